// Radius search and k-NN over a CGA (the Eq. 8 set generalised): every
// stored voxel within a squared integer distance r2 of each query voxel in
// ascending CGA index, or the k least (distance^2, key) in ascending order.
//   k_radius_count  one warp per query: the slabs whose x lies within the
//                   radius are shared 32 at a time among the lanes; a lane
//                   walks its slab's columns inside the circle left for y and
//                   counts each column's z interval by two searches
//   k_scan_*        exclusive prefix of the counts (64-bit offsets)
//   k_radius_fill   the same walk; per group of 32 slabs a warp scan of the
//                   lanes' counts places every slab's voxels, so the output
//                   is in (x, y, z) = CGA order without sorting
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "k_common.cuh"

// Blocks per SM the search kernels are compiled for (their register budgets;
// measured on GB300: 5 or 6 blocks were no faster for either kernel).
#ifndef CGA_KNN_BLOCKS
#define CGA_KNN_BLOCKS 4
#endif
#ifndef CGA_RADIUS_BLOCKS
#define CGA_RADIUS_BLOCKS 1
#endif

namespace libcga {

namespace {

// Largest s with s * s <= v (v < 2^63).  Below 2^46 a single-precision
// estimate is within 2 of the root (the rounding of v to float moves the
// root by at most a quarter, sqrtf's own rounding by at most half a unit of
// a number below 2^23), so two exact integer steps at most fix it; the rare
// larger arguments take the double-precision estimate, which GB300 runs at a
// small fraction of the single-precision rate.
__device__ __forceinline__ unsigned long long isqrt_u64(unsigned long long v) {
  unsigned long long s = v < (1ull << 46) ? (unsigned long long)sqrtf((float)v)
                                          : (unsigned long long)sqrt((double)v);
  while (s > 0 && s * s > v) --s;
  while ((s + 1) * (s + 1) <= v) ++s;
  return s;
}

// |v - q| of a stored coordinate and a query coordinate (clamped to
// +-2^30, so the difference fits 31 bits).
__device__ __forceinline__ uint32_t absdiff32(uint32_t v, int q) {
  const int d = (int)v - q;
  return (uint32_t)(d < 0 ? -d : d);
}

__device__ __forceinline__ unsigned long long sq(uint32_t d) {
  return (unsigned long long)d * d;
}

// The grid coordinates [lo, hi] within reach of q on one axis, where rem is
// the squared distance left for it: [q - isqrt(rem), q + isqrt(rem)] cut to
// [0, top] (in 64 bits: the reach may exceed 2^31).  False when empty.
__device__ __forceinline__ bool axis_window(int q, unsigned long long rem, int top, int& lo,
                                            int& hi) {
  const long long r = (long long)isqrt_u64(rem);
  const long long l = (long long)q - r, h = (long long)q + r;
  if (h < 0 || l > top) return false;
  lo = (int)max(l, 0ll);
  hi = (int)min(h, (long long)top);
  return true;
}


struct RQuery {
  int x, y, z;  // query voxel (clamped only to +-2^30)
  bool valid;
};

__device__ __forceinline__ RQuery radius_query(const SearchSeg& sg, uint32_t j) {
  const float* p = sg.q + 3 * (size_t)j;
  const float px = __ldg(p), py = __ldg(p + 1), pz = __ldg(p + 2);
  RQuery q;
  q.valid = isfinite(px) && isfinite(py) && isfinite(pz);
  q.x = q.valid ? (int)quantize_query(px, sg.scale, sg.off[0]) : 0;
  q.y = q.valid ? (int)quantize_query(py, sg.scale, sg.off[1]) : 0;
  q.z = q.valid ? (int)quantize_query(pz, sg.scale, sg.off[2]) : 0;
  return q;
}

// Column c's voxel range [zs, ze) and z range [zlo, zhi]: one load from the
// column table when there is one, else the range is taken as the whole axis
// (so every shortcut below falls back to a search).
__device__ __forceinline__ void column_of(const Levels& a, const uint4* ctab, uint32_t c,
                                          uint32_t& zs, uint32_t& ze, uint32_t& zlo,
                                          uint32_t& zhi) {
  if (ctab != nullptr) {
    const uint4 e = __ldg(ctab + c);
    zs = e.x;
    ze = e.y;
    zlo = e.z & 0xffffu;
    zhi = e.z >> 16;
  } else {
    zs = __ldg(a.ptr1 + c);
    ze = __ldg(a.ptr1 + c + 1);
    zlo = 0;
    zhi = 0xffffu;
  }
}

// Slabs [s0, s1) of a whose x lies within the radius of the query.
__device__ __forceinline__ void radius_slabs(const Levels& a, uint32_t h, const RQuery& q,
                                             unsigned long long r2, uint32_t& s0, uint32_t& s1) {
  s0 = s1 = 0;
  if (!q.valid || h == 0) return;
  int lo, hi;
  if (!axis_window(q.x, r2, (1 << a.bits) - 1, lo, hi)) return;
  s0 = lower_bound_u16(a.idx2, 0, h, (uint32_t)lo);
  s1 = lower_bound_u16(a.idx2, s0, h, (uint32_t)hi + 1);
}

// Count (EMIT = false) or write in (y, z) order from position `pos` (EMIT =
// true) the voxels of one slab within the radius; returns the count.
template <bool EMIT>
__device__ __forceinline__ unsigned long long radius_slab(const Levels& a, const uint4* ctab,
                                                          uint32_t slab,
                                                          const RQuery& q, unsigned long long r2,
                                                          uint32_t* idx, unsigned long long* d2,
                                                          unsigned long long pos) {
  const int top = (1 << a.bits) - 1;
  const uint32_t x = __ldg(a.idx2 + slab);
  const unsigned long long dx2 = sq(absdiff32(x, q.x));
  if (dx2 > r2) return 0;
  int ylo, yhi;
  if (!axis_window(q.y, r2 - dx2, top, ylo, yhi)) return 0;
  const uint32_t ys = __ldg(a.ptr2 + slab), ye = __ldg(a.ptr2 + slab + 1);
  unsigned long long n = 0;
  for (uint32_t c = lower_bound_u16(a.idx1, ys, ye, (uint32_t)ylo); c < ye; ++c) {
    const uint32_t y = __ldg(a.idx1 + c);
    if ((int)y > yhi) break;
    const unsigned long long dxy = dx2 + sq(absdiff32(y, q.y));
    int zlo, zhi;
    if (!axis_window(q.z, r2 - dxy, top, zlo, zhi)) continue;
    uint32_t zs, ze, clo, chi;
    column_of(a, ctab, c, zs, ze, clo, chi);
    if ((uint32_t)zhi < clo || (uint32_t)zlo > chi) continue;
    const uint32_t p0 = (uint32_t)zlo <= clo ? zs : lower_bound_u16(a.idx0, zs, ze, (uint32_t)zlo);
    const uint32_t p1 =
        (uint32_t)zhi >= chi ? ze : lower_bound_u16(a.idx0, p0, ze, (uint32_t)zhi + 1);
    if (EMIT) {
      for (uint32_t p = p0; p < p1; ++p) {
        const unsigned long long dz = absdiff32(__ldg(a.idx0 + p), q.z);
        idx[pos + n + (p - p0)] = p;
        d2[pos + n + (p - p0)] = dxy + dz * dz;
      }
    }
    n += p1 - p0;
  }
  return n;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Query of slot `slot`: the slot itself, or the index in the low 32 bits of
// the Morton-ordered key when an order is given (neighbouring warps then
// search neighbouring space and share the cache).
__device__ __forceinline__ uint32_t slot_query(const unsigned long long* order, uint32_t slot) {
  return order != nullptr ? (uint32_t)__ldg(order + slot) : slot;
}

__global__ void __launch_bounds__(256, CGA_RADIUS_BLOCKS) k_radius_count(SearchSeg sg, unsigned long long r2,
                               const unsigned long long* __restrict__ order,
                               unsigned long long* counts) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t h = (uint32_t)sg.a.hdr->cnt[2];
  for (uint32_t sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < sg.m; sl += nw) {
    const uint32_t j = slot_query(order, sl);
    const RQuery q = radius_query(sg, j);
    uint32_t s0, s1;
    radius_slabs(sg.a, h, q, r2, s0, s1);
    unsigned long long n = 0;
    for (uint32_t s = s0 + lane; s < s1; s += 32) {
      n += radius_slab<false>(sg.a, sg.ctab, s, q, r2, nullptr, nullptr, 0);
    }
    n = warp_sum_u64(n);
    if (lane == 0) counts[j] = n;
  }
}

__global__ void __launch_bounds__(256, CGA_RADIUS_BLOCKS) k_radius_fill(SearchSeg sg, unsigned long long r2,
                              const unsigned long long* __restrict__ order,
                              const unsigned long long* __restrict__ offsets, uint32_t* idx,
                              unsigned long long* d2) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t h = (uint32_t)sg.a.hdr->cnt[2];
  for (uint32_t sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < sg.m; sl += nw) {
    const uint32_t j = slot_query(order, sl);
    const RQuery q = radius_query(sg, j);
    uint32_t s0, s1;
    radius_slabs(sg.a, h, q, r2, s0, s1);
    unsigned long long base = offsets[j];
    for (uint32_t g = s0; g < s1; g += 32) {
      const uint32_t s = g + lane;
      const unsigned long long n =
          s < s1 ? radius_slab<false>(sg.a, sg.ctab, s, q, r2, nullptr, nullptr, 0) : 0ull;
      unsigned long long inc = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += t;
      }
      if (n > 0) radius_slab<true>(sg.a, sg.ctab, s, q, r2, idx, d2, base + inc - n);
      base += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
}

// Exclusive scan of v[0, m) in place, v[m] = total: B blocks, each owning a
// contiguous chunk; block totals are scanned by one block, then each chunk
// is rescanned with its prefix.
__global__ void k_scan_totals(const unsigned long long* v, uint64_t m, uint64_t chunk,
                              unsigned long long* totals) {
  __shared__ unsigned long long s_warp[kWarps];
  const uint64_t lo = blockIdx.x * chunk, hi = min(lo + chunk, m);
  unsigned long long t = 0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += kThreads) t += v[i];
  unsigned long long tot;
  block_excl_scan(t, tot, s_warp);
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void k_scan_top(unsigned long long* totals, uint32_t B) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long run = 0;
  for (uint32_t b = 0; b < B; ++b) {
    const unsigned long long t = totals[b];
    totals[b] = run;
    run += t;
  }
  totals[B] = run;
}

__global__ void k_scan_apply(unsigned long long* v, uint64_t m, uint64_t chunk,
                             const unsigned long long* totals, uint32_t B) {
  __shared__ unsigned long long s_warp[kWarps];
  const uint64_t lo = blockIdx.x * chunk, hi = min(lo + chunk, m);
  unsigned long long run = totals[blockIdx.x];
  for (uint64_t b0 = lo; b0 < hi; b0 += kThreads) {
    const uint64_t i = b0 + threadIdx.x;
    const unsigned long long x = i < hi ? v[i] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan(x, tot, s_warp);
    if (i < hi) v[i] = run + ex;
    run += tot;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) v[m] = totals[B];
}

// ---- k nearest -------------------------------------------------------------
// The warp's list of the k best (distance^2, index) so far, lane i holding
// the i-th; lanes >= k hold the sentinel (~0, ~0).  The CGA index of a voxel
// rises with its key, so (distance^2, index) order is (distance^2, key) order.
struct TopK {
  unsigned long long d2;
  uint32_t idx;
};

__device__ __forceinline__ bool pair_less(unsigned long long da, uint32_t ia,
                                          unsigned long long db, uint32_t ib) {
  return da < db || (da == db && ia < ib);
}

// Offer one candidate (the same in every lane): it enters before the first
// entry that is not below it, the entries after it move up one lane and the
// k-th falls out.
__device__ __forceinline__ void topk_insert(TopK& t, uint32_t lane, uint32_t k,
                                            unsigned long long cd, uint32_t ci) {
  const bool before = lane < k && pair_less(t.d2, t.idx, cd, ci);
  const uint32_t pos = __popc(__ballot_sync(0xffffffffu, before));
  const unsigned long long ud = __shfl_up_sync(0xffffffffu, t.d2, 1);
  const uint32_t ui = __shfl_up_sync(0xffffffffu, t.idx, 1);
  if (pos < k) {
    if (lane == pos) {
      t.d2 = cd;
      t.idx = ci;
    } else if (lane > pos && lane < k) {
      t.d2 = ud;
      t.idx = ui;
    }
  }
}

// One compare-exchange step of a bitonic network across the warp: the pair
// (lane, lane ^ j) is put in ascending order when `up`, descending otherwise.
__device__ __forceinline__ void bitonic_step(unsigned long long& d, uint32_t& i, uint32_t lane,
                                             uint32_t j, bool up) {
  const unsigned long long od = __shfl_xor_sync(0xffffffffu, d, j);
  const uint32_t oi = __shfl_xor_sync(0xffffffffu, i, j);
  const bool keep_min = ((lane & j) == 0) == up;
  const bool take = keep_min ? pair_less(od, oi, d, i) : pair_less(d, i, od, oi);
  if (take) {
    d = od;
    i = oi;
  }
}

// Offer every lane's candidate at once (sentinel where a lane has none): the
// candidates are sorted by a bitonic network, the lane-wise minimum of the
// list and the reversed candidates holds the 32 least of both as a bitonic
// sequence, and a bitonic merge orders it.
__device__ __forceinline__ void topk_insert_all(TopK& t, uint32_t lane, uint32_t k,
                                                unsigned long long cd, uint32_t ci) {
#pragma unroll
  for (uint32_t w = 2; w <= 32; w <<= 1) {
#pragma unroll
    for (uint32_t j = w >> 1; j > 0; j >>= 1) bitonic_step(cd, ci, lane, j, (lane & w) == 0);
  }
  const unsigned long long rd = __shfl_sync(0xffffffffu, cd, 31 - lane);
  const uint32_t ri = __shfl_sync(0xffffffffu, ci, 31 - lane);
  if (pair_less(rd, ri, t.d2, t.idx)) {
    t.d2 = rd;
    t.idx = ri;
  }
#pragma unroll
  for (uint32_t j = 16; j > 0; j >>= 1) bitonic_step(t.d2, t.idx, lane, j, true);
  if (lane >= k) {
    t.d2 = ~0ull;
    t.idx = 0xffffffffu;
  }
}

// Above this many candidates in one step, one bitonic merge is cheaper than
// inserting them one by one.
constexpr int kKnnBatch = 8;
constexpr uint32_t kKnnLargeThreads = 128;  // 4 warps, each with its own buffer

// Candidate collection for k <= 32: the list in registers.
struct RegList {
  TopK t;
  uint32_t k;

  __device__ __forceinline__ void init(uint32_t kk) {
    t = TopK{~0ull, 0xffffffffu};
    k = kk;
  }
  // Offer each lane's candidate (if any); returns the new pruning bound.
  __device__ __forceinline__ unsigned long long offer(bool has, unsigned long long cd, uint32_t ci,
                                                      uint32_t lane) {
    uint32_t pending = __ballot_sync(0xffffffffu, has);
    if (__popc(pending) > kKnnBatch) {
      topk_insert_all(t, lane, k, cd, ci);
    } else {
      while (pending) {
        const uint32_t src = __ffs(pending) - 1;
        pending &= pending - 1;
        topk_insert(t, lane, k, __shfl_sync(0xffffffffu, cd, src),
                    __shfl_sync(0xffffffffu, ci, src));
      }
    }
    return __shfl_sync(0xffffffffu, t.d2, k - 1);
  }
  __device__ __forceinline__ void finish(uint32_t lane, size_t row, uint32_t* out_idx,
                                         unsigned long long* out_d2) {
    if (lane < k) {
      out_idx[row + lane] = t.idx;
      out_d2[row + lane] = t.d2;
    }
  }
};

// Candidate collection for 32 < k <= CGA_KNN_MAX_K: the warp's buffer of
// `cap` (a power of two, at least 2k) entries in shared memory.  Candidates
// are appended unsorted; whenever the next step could overflow it, or when it
// first holds k, the k-th least distance B is found by bisection on the count
// of entries at most a trial value, every entry beyond B is dropped, and B
// becomes the bound (if ties at B leave too little room, the buffer is
// sorted by a bitonic network and cut to exactly k instead).  Every voxel
// pruned by a bound is beaten by k collected ones, so the final sort's first
// k are the answer.
struct SmemList {
  unsigned long long* d;
  uint32_t* ix;
  uint32_t n, k, cap;

  __device__ __forceinline__ void sort_cut(uint32_t lane) {
    uint32_t P = 32;
    while (P < n) P <<= 1;
    for (uint32_t e = n + lane; e < P; e += 32) {
      d[e] = ~0ull;
      ix[e] = 0xffffffffu;
    }
    __syncwarp();
    for (uint32_t w = 2; w <= P; w <<= 1) {
      for (uint32_t jj = w >> 1; jj > 0; jj >>= 1) {
        for (uint32_t tt = lane; tt < P / 2; tt += 32) {
          const uint32_t i = ((tt & ~(jj - 1)) << 1) | (tt & (jj - 1)), l = i + jj;
          const unsigned long long di = d[i], dl = d[l];
          const uint32_t xi = ix[i], xl = ix[l];
          const bool up = (i & w) == 0;
          if (up ? pair_less(dl, xl, di, xi) : pair_less(di, xi, dl, xl)) {
            d[i] = dl;
            ix[i] = xl;
            d[l] = di;
            ix[l] = xi;
          }
        }
        __syncwarp();
      }
    }
    n = min(n, k);
  }
  // Keep the entries of distance at most B, the k-th least; returns B.
  __device__ __forceinline__ unsigned long long select_cut(uint32_t lane) {
    unsigned long long lo = ~0ull, hi = 0;
    for (uint32_t e = lane; e < n; e += 32) {
      lo = min(lo, d[e]);
      hi = max(hi, d[e]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    while (lo < hi) {
      const unsigned long long mid = lo + ((hi - lo) >> 1);
      uint32_t c = 0;
      for (uint32_t e = lane; e < n; e += 32) c += d[e] <= mid ? 1u : 0u;
      if (__reduce_add_sync(0xffffffffu, c) >= k) hi = mid; else lo = mid + 1;
    }
    uint32_t out = 0;
    for (uint32_t base = 0; base < n; base += 32) {
      const uint32_t e = base + lane;
      const bool keep = e < n && d[e] <= lo;
      const unsigned long long dv = keep ? d[e] : 0ull;
      const uint32_t xv = keep ? ix[e] : 0u;
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) {
        const uint32_t p = out + __popc(bal & ((1u << lane) - 1u));
        d[p] = dv;
        ix[p] = xv;
      }
      out += __popc(bal);
      __syncwarp();
    }
    n = out;
    if (n + 32 > cap) sort_cut(lane);  // too many ties at B: cut to exactly k
    return lo;
  }
  __device__ __forceinline__ void init(uint32_t kk, uint32_t cp, unsigned long long* dd,
                                       uint32_t* xx) {
    d = dd;
    ix = xx;
    n = 0;
    k = kk;
    cap = cp;
  }
  __device__ __forceinline__ unsigned long long offer(bool has, unsigned long long cd, uint32_t ci,
                                                      uint32_t lane, unsigned long long bound) {
    const uint32_t pending = __ballot_sync(0xffffffffu, has);
    if (has) {
      const uint32_t pos = n + __popc(pending & ((1u << lane) - 1u));
      d[pos] = cd;
      ix[pos] = ci;
    }
    n += __popc(pending);
    __syncwarp();
    if (n + 32 > cap || (bound == ~0ull && n >= k)) return select_cut(lane);
    return bound;
  }
  __device__ __forceinline__ void finish(uint32_t lane, size_t row, uint32_t* out_idx,
                                         unsigned long long* out_d2) {
    sort_cut(lane);
    for (uint32_t e = lane; e < k; e += 32) {
      out_idx[row + e] = e < n ? ix[e] : 0xffffffffu;
      out_d2[row + e] = e < n ? d[e] : ~0ull;
    }
    __syncwarp();
  }
};

// k nearest of one query, one warp: slab rounds as in the NN search (16 per
// side), every lane walking its slab's columns nearest-first in y and each
// column's voxels nearest-first in z.  The lanes step in lockstep, each step
// offering at most one candidate per lane, so that the candidates enter the
// list together and the k-th distance prunes every walk; a lane whose column
// runs out moves to its next column (and offers that column's nearest voxel)
// in the same step.
template <bool LARGE>
__global__ void __launch_bounds__(LARGE ? kKnnLargeThreads : 256, LARGE ? 1 : CGA_KNN_BLOCKS)
    k_knn(SearchSeg sg, uint32_t k, uint32_t cap, const unsigned long long* __restrict__ order,
          uint32_t* out_idx, unsigned long long* out_d2) {
  extern __shared__ unsigned long long s_knn[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const Levels& a = sg.a;
  const uint32_t u = (uint32_t)a.hdr->cnt[0], h = (uint32_t)a.hdr->cnt[2];
  const int top = (1 << a.bits) - 1;
  typename std::conditional<LARGE, SmemList, RegList>::type list;
  for (uint32_t sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < sg.m; sl += nw) {
    const uint32_t j = slot_query(order, sl);
    if constexpr (LARGE) {
      const uint32_t wb = threadIdx.x >> 5;
      unsigned long long* base = s_knn + (size_t)wb * cap;
      list.init(k, cap, base,
                reinterpret_cast<uint32_t*>(s_knn + (size_t)(blockDim.x >> 5) * cap) + (size_t)wb * cap);
    } else {
      list.init(k);
    }
    const RQuery q = radius_query(sg, j);
    if (q.valid && u > 0) {
      const int qx = q.x, qy = q.y, qz = q.z;
      const uint32_t cqy = (uint32_t)min(max(qy, 0), top);
      const uint32_t cqz = (uint32_t)min(max(qz, 0), top);
      const uint32_t xr0 = lower_bound_u16(a.idx2, 0, h, (uint32_t)min(max(qx, 0), top));
      const bool right = (lane & 1u) == 0u;
      unsigned long long bound = ~0ull;
      for (uint32_t r = 0;; ++r) {
        const int kk = (int)(r * 16u + (lane >> 1));
        const int slab = right ? (int)xr0 + kk : (int)xr0 - 1 - kk;
        bool work = slab >= 0 && slab < (int)h;
        unsigned long long dx2 = 0;
        uint32_t ys = 0, ye = 0;
        if (work) {
          dx2 = sq(absdiff32(__ldg(a.idx2 + slab), qx));
          ys = __ldg(a.ptr2 + slab);
          ye = __ldg(a.ptr2 + slab + 1);
          work = dx2 <= bound;
        }
        if (!__any_sync(0xffffffffu, work)) break;
        // column cursors outward from the query's y: [cr, ye) to the right,
        // [ys, cl) to the left; z cursors likewise within the column
        uint32_t cr = 0, cl = 0;
        if (work) {
          cr = lower_bound_u16(a.idx1, ys, ye, cqy);
          cl = cr;
        }
        bool in_col = false;
        unsigned long long dxy = 0;
        uint32_t zs = 0, ze = 0, zu = 0, zd = 0;
        while (__any_sync(0xffffffffu, work)) {
          bool has = false;
          unsigned long long cd = ~0ull;
          uint32_t ci = 0xffffffffu;
#pragma unroll 1
          for (int pass = 0; pass < 2; ++pass) {
            if (work && !has && !in_col) {
              // the next column, nearest in y first, while it can still beat the bound
              const bool hr = cr < ye, hl = cl > ys;
              const uint32_t er = hr ? absdiff32(__ldg(a.idx1 + cr), qy) : 0xffffffffu;
              const uint32_t el = hl ? absdiff32(__ldg(a.idx1 + cl - 1), qy) : 0xffffffffu;
              const bool gr = hr && (!hl || er <= el);
              const unsigned long long d = dx2 + sq(gr ? er : el);
              if ((!hr && !hl) || d > bound) {
                work = false;
              } else {
                const uint32_t c = gr ? cr++ : --cl;
                dxy = d;
                uint32_t clo, chi;
                column_of(a, sg.ctab, c, zs, ze, clo, chi);
                zu = cqz <= clo ? zs : (cqz > chi ? ze : lower_bound_u16(a.idx0, zs, ze, cqz));
                zd = zu;
                in_col = true;
              }
            }
            if (work && !has && in_col) {
              // the column's next voxel, nearest in z first
              const bool hu = zu < ze, hd = zd > zs;
              const uint32_t eu = hu ? absdiff32(__ldg(a.idx0 + zu), qz) : 0xffffffffu;
              const uint32_t ed = hd ? absdiff32(__ldg(a.idx0 + zd - 1), qz) : 0xffffffffu;
              const bool gu = hu && (!hd || eu <= ed);
              const unsigned long long d = dxy + sq(gu ? eu : ed);
              if ((!hu && !hd) || d > bound) {
                in_col = false;
              } else {
                ci = gu ? zu++ : --zd;
                cd = d;
                has = true;
              }
            }
          }
          if constexpr (LARGE) {
            bound = list.offer(has, cd, ci, lane, bound);
          } else {
            bound = list.offer(has, cd, ci, lane);
          }
        }
      }
    }
    list.finish(lane, (size_t)j * k, out_idx, out_d2);
  }
}

unsigned search_blocks(uint64_t m) {
  return (unsigned)std::min<uint64_t>((std::max<uint64_t>(m, 1) + 7) / 8,
                                      (uint64_t)device_sm_count() * 8);
}

}  // namespace

// Buffer entries per warp for k > 32: the least power of two >= 2k.
static uint32_t knn_cap(uint32_t k) {
  uint32_t c = 64;
  while (c < 2 * k) c <<= 1;
  return c;
}

cudaError_t run_knn(const SearchSeg& sg, uint32_t k, const unsigned long long* order, uint32_t* idx,
                    unsigned long long* d2, cudaStream_t stream) {
  if (sg.m == 0) return cudaSuccess;
  if (k <= 32) {
    k_knn<false><<<search_blocks(sg.m), 256, 0, stream>>>(sg, k, 0, order, idx, d2);
  } else {
    const uint32_t cap = knn_cap(k);
    const size_t smem = (size_t)(kKnnLargeThreads / 32) * cap * 12;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
      attr = cudaFuncSetAttribute(k_knn<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)((kKnnLargeThreads / 32) * knn_cap(kKnnMaxK) * 12));
    });
    if (attr != cudaSuccess) return attr;
    const unsigned blocks = (unsigned)std::min<uint64_t>((sg.m + 3) / 4,
                                                         (uint64_t)device_sm_count() * 4);
    k_knn<true><<<blocks, kKnnLargeThreads, smem, stream>>>(sg, k, cap, order, idx, d2);
  }
  count_launch(1);
  return cudaGetLastError();
}

size_t radius_scratch_bytes() { return 1025 * sizeof(unsigned long long); }

cudaError_t run_radius_count(const SearchSeg& sg, unsigned long long r2,
                             const unsigned long long* order, unsigned long long* offsets,
                             void* scratch, cudaStream_t stream) {
  unsigned long long* totals = static_cast<unsigned long long*>(scratch);
  if (sg.m > 0) {
    k_radius_count<<<search_blocks(sg.m), 256, 0, stream>>>(sg, r2, order, offsets);
  }
  const uint32_t B = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(1024, (sg.m + 4095) / 4096));
  const uint64_t chunk = (sg.m + B - 1) / B;
  k_scan_totals<<<B, kThreads, 0, stream>>>(offsets, sg.m, std::max<uint64_t>(chunk, 1), totals);
  k_scan_top<<<1, 32, 0, stream>>>(totals, B);
  k_scan_apply<<<B, kThreads, 0, stream>>>(offsets, sg.m, std::max<uint64_t>(chunk, 1), totals, B);
  count_launch(sg.m > 0 ? 4 : 3);
  return cudaGetLastError();
}

cudaError_t run_radius_fill(const SearchSeg& sg, unsigned long long r2,
                            const unsigned long long* order, const unsigned long long* offsets,
                            uint32_t* idx, unsigned long long* d2, cudaStream_t stream) {
  if (sg.m == 0) return cudaSuccess;
  k_radius_fill<<<search_blocks(sg.m), 256, 0, stream>>>(sg, r2, order, offsets, idx, d2);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace libcga
