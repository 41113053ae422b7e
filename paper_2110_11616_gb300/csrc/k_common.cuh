// Device helpers shared by the libcga kernels: relaxed flag access, bounded
// decoupled look-back, block scans, and searches over the CGA arrays.
#pragma once
#include "cga_impl.h"

namespace libcga {

constexpr uint32_t kFlagAgg = 1u << 30;   // tile aggregate published
constexpr uint32_t kFlagInc = 2u << 30;   // inclusive prefix published
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr uint32_t kSpinLimit = 1u << 22;  // polls of one look-back word
constexpr uint32_t kErrInternal = 4u;      // a device consistency check failed

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // one second per word

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Decoupled look-back over the tiles (first, tile) of one segment.  Each
// tile publishes one 32-bit word per counter: 2 flag bits + a 30-bit value.
// Tile ids are handed out in launch order by an atomic counter, so every
// predecessor is already resident and the wait ends; it is still bounded: after
// kSpinLimit polls, or one second, on one word the error bit is set and the
// wait stops.
__device__ __forceinline__ uint32_t lookback(const uint32_t* look, uint32_t stride, uint32_t tile,
                                             uint32_t first, unsigned int* err) {
  uint32_t excl = 0;
  uint32_t j = tile;
  while (j > first) {
    --j;
    uint32_t v;
    uint32_t spins = 0;
    unsigned long long t0 = 0;
    while (true) {
      v = ld_relaxed(look + (size_t)j * stride);
      if (v & (kFlagAgg | kFlagInc)) break;
      ++spins;
      if (spins == 32) t0 = global_ns();
      if (spins > kSpinLimit || (spins > 32 && (spins & 63) == 0 && global_ns() - t0 > kWaitLimitNs)) {
        atomicOr(err, kErrTimeout);
        return excl;
      }
      if (spins > 32) __nanosleep(100);
    }
    excl += v & kValMask;
    if (v & kFlagInc) break;
  }
  return excl;
}

// One axis of the grid (Sec. II-E-2-a box): floorf(fmaf(v, scale, off))
// clamped in float to [0, hi].
__device__ __forceinline__ uint32_t quantize_axis(float v, float scale, float off, float hi) {
  float f = floorf(__fmaf_rn(v, scale, off));
  f = fminf(fmaxf(f, 0.0f), hi);
  return (uint32_t)f;
}

// Query voxel coordinate of an NN / radius / k-NN search: floorf(fmaf(v,
// scale, off)) clamped only to [-2^30, 2^30] (queries outside the box keep
// their true distance).
__device__ __forceinline__ long long quantize_query(float v, float scale, float off) {
  float f = floorf(__fmaf_rn(v, scale, off));
  f = fminf(fmaxf(f, -1073741824.0f), 1073741824.0f);
  return (long long)f;
}

// Voxel key x << 2b | y << b | z of one point, after the rigid transform X
// (R row-major, then t) by the fixed fmaf nesting when has_x.  False for a
// non-finite point or transform result (key left 0).
template <typename K>
__device__ __forceinline__ bool point_key(float x, float y, float z, bool has_x, const float* X,
                                          float scale, const float* off, uint32_t b, K& key) {
  bool ok = isfinite(x) && isfinite(y) && isfinite(z);
  if (has_x) {
    const float x2 = __fmaf_rn(X[0], x, __fmaf_rn(X[1], y, __fmaf_rn(X[2], z, X[9])));
    const float y2 = __fmaf_rn(X[3], x, __fmaf_rn(X[4], y, __fmaf_rn(X[5], z, X[10])));
    const float z2 = __fmaf_rn(X[6], x, __fmaf_rn(X[7], y, __fmaf_rn(X[8], z, X[11])));
    x = x2;
    y = y2;
    z = z2;
    ok = ok && isfinite(x) && isfinite(y) && isfinite(z);
  }
  key = 0;
  if (!ok) return false;
  const float hi = (float)((1u << b) - 1u);
  const uint32_t qx = quantize_axis(x, scale, off[0], hi);
  const uint32_t qy = quantize_axis(y, scale, off[1], hi);
  const uint32_t qz = quantize_axis(z, scale, off[2], hi);
  key = ((K)qx << (2 * b)) | ((K)qy << b) | (K)qz;
  return true;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan across a kThreads block.  s_warp: kWarps scratch words.
// Contains two __syncthreads.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T& total, T* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  T before = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) {
    T x = s_warp[i];
    if (i < w) before += x;
    tot += x;
  }
  __syncthreads();
  total = tot;
  return before + inc - v;
}

// Largest c in [lo, hi] with ptr[c] <= p (requires ptr[lo] <= p).
__device__ __forceinline__ uint32_t search_le(const uint32_t* __restrict__ ptr, uint32_t lo,
                                              uint32_t hi, uint32_t p) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(ptr + mid) <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// First index in [lo, hi) whose value is >= v (hi when none).
__device__ __forceinline__ uint32_t lower_bound_u16(const uint16_t* __restrict__ a, uint32_t lo,
                                                    uint32_t hi, uint32_t v) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((uint32_t)__ldg(a + mid) < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// search_le by one whole warp: each round the 32 lanes probe 32 evenly
// spaced entries of the remaining range, so a range of n entries takes about
// log32(n) dependent loads instead of log2(n).  Every lane returns the result.
__device__ __forceinline__ uint32_t warp_search_le(const uint32_t* __restrict__ ptr, uint32_t lo,
                                                   uint32_t hi, uint32_t p) {
  const uint32_t lane = threadIdx.x & 31;
  while (hi - lo >= 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t probe = min(lo + step * (lane + 1), hi);
    const uint32_t k = __popc(__ballot_sync(0xffffffffu, __ldg(ptr + probe) <= p));
    const uint32_t nlo = min(lo + step * k, hi);
    const uint32_t nhi = k == 32 ? hi : min(lo + step * (k + 1), hi) - 1;
    lo = nlo;
    hi = nhi;
  }
  const bool le = lo + lane <= hi && __ldg(ptr + lo + lane) <= p;
  return lo + __popc(__ballot_sync(0xffffffffu, le)) - 1;
}

// key_at by one whole warp.
__device__ __forceinline__ unsigned long long warp_key_at(const Levels& a, uint32_t g, uint32_t h,
                                                          uint32_t p) {
  const uint32_t b = a.bits;
  const uint32_t c = warp_search_le(a.ptr1, 0, g - 1, p);
  const uint32_t xr = warp_search_le(a.ptr2, 0, h - 1, c);
  return ((unsigned long long)__ldg(a.idx2 + xr) << (2 * b)) |
         ((unsigned long long)__ldg(a.idx1 + c) << b) | (unsigned long long)__ldg(a.idx0 + p);
}

// lower_bound_u16 by one whole warp (32 probes per round).
__device__ __forceinline__ uint32_t warp_lower_bound_u16(const uint16_t* __restrict__ a,
                                                         uint32_t lo, uint32_t hi, uint32_t v) {
  const uint32_t lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t probe = min(lo + step * (lane + 1), hi) - 1;
    const uint32_t k = __popc(__ballot_sync(0xffffffffu, (uint32_t)__ldg(a + probe) < v));
    if (k == 32) return hi;
    const uint32_t nhi = min(lo + step * (k + 1), hi);
    if (k > 0) lo = lo + step * k;
    hi = nhi;
  }
  const bool lt = lo + lane < hi && (uint32_t)__ldg(a + lo + lane) < v;
  return lo + __popc(__ballot_sync(0xffffffffu, lt));
}

// Key of the point at CGA position p (p < u).  g, h: level sizes.
__device__ __forceinline__ unsigned long long key_at(const Levels& a, uint32_t g, uint32_t h,
                                                     uint32_t p) {
  const uint32_t b = a.bits;
  const uint32_t c = search_le(a.ptr1, 0, g - 1, p);
  const uint32_t xr = search_le(a.ptr2, 0, h - 1, c);
  return ((unsigned long long)__ldg(a.idx2 + xr) << (2 * b)) |
         ((unsigned long long)__ldg(a.idx1 + c) << b) | (unsigned long long)__ldg(a.idx0 + p);
}

// Number of stored keys smaller than `key`: the Sec. V-A lookup (x in
// X_index, then y in its Y range, then z in its column) in lower-bound form.
__device__ __forceinline__ uint32_t rank_of(const Levels& a, uint32_t h, unsigned long long key) {
  const uint32_t b = a.bits, m = (1u << b) - 1u;
  const uint32_t x = (uint32_t)(key >> (2 * b)), y = (uint32_t)(key >> b) & m,
                 z = (uint32_t)key & m;
  const uint32_t xr = lower_bound_u16(a.idx2, 0, h, x);
  if (xr == h || __ldg(a.idx2 + xr) != x) return __ldg(a.ptr1 + __ldg(a.ptr2 + xr));
  const uint32_t ys = __ldg(a.ptr2 + xr), ye = __ldg(a.ptr2 + xr + 1);
  const uint32_t c = lower_bound_u16(a.idx1, ys, ye, y);
  if (c == ye || __ldg(a.idx1 + c) != y) return __ldg(a.ptr1 + c);
  return lower_bound_u16(a.idx0, __ldg(a.ptr1 + c), __ldg(a.ptr1 + c + 1), z);
}

// rank_of by one whole warp; *found tells whether `key` itself is stored.
__device__ __forceinline__ uint32_t warp_rank_of(const Levels& a, uint32_t h,
                                                 unsigned long long key, bool* found) {
  const uint32_t b = a.bits, m = (1u << b) - 1u;
  const uint32_t x = (uint32_t)(key >> (2 * b)), y = (uint32_t)(key >> b) & m,
                 z = (uint32_t)key & m;
  *found = false;
  const uint32_t xr = warp_lower_bound_u16(a.idx2, 0, h, x);
  if (xr == h || __ldg(a.idx2 + xr) != x) return __ldg(a.ptr1 + __ldg(a.ptr2 + xr));
  const uint32_t ys = __ldg(a.ptr2 + xr), ye = __ldg(a.ptr2 + xr + 1);
  const uint32_t c = warp_lower_bound_u16(a.idx1, ys, ye, y);
  if (c == ye || __ldg(a.idx1 + c) != y) return __ldg(a.ptr1 + c);
  const uint32_t zs = __ldg(a.ptr1 + c), ze = __ldg(a.ptr1 + c + 1);
  const uint32_t zr = warp_lower_bound_u16(a.idx0, zs, ze, z);
  *found = zr < ze && __ldg(a.idx0 + zr) == z;
  return zr;
}

// rank_of, and whether `key` itself is stored (then the rank is its index).
__device__ __forceinline__ uint32_t rank_of_found(const Levels& a, uint32_t h,
                                                  unsigned long long key, bool& found) {
  const uint32_t b = a.bits, m = (1u << b) - 1u;
  const uint32_t x = (uint32_t)(key >> (2 * b)), y = (uint32_t)(key >> b) & m,
                 z = (uint32_t)key & m;
  found = false;
  const uint32_t xr = lower_bound_u16(a.idx2, 0, h, x);
  if (xr == h || __ldg(a.idx2 + xr) != x) return __ldg(a.ptr1 + __ldg(a.ptr2 + xr));
  const uint32_t ys = __ldg(a.ptr2 + xr), ye = __ldg(a.ptr2 + xr + 1);
  const uint32_t c = lower_bound_u16(a.idx1, ys, ye, y);
  if (c == ye || __ldg(a.idx1 + c) != y) return __ldg(a.ptr1 + c);
  const uint32_t zs = __ldg(a.ptr1 + c), ze = __ldg(a.ptr1 + c + 1);
  const uint32_t zr = lower_bound_u16(a.idx0, zs, ze, z);
  found = zr < ze && __ldg(a.idx0 + zr) == z;
  return zr;
}

// Column and x windows of the CGA positions [p0, p1] (inclusive, p1 < u).
struct Window {
  uint32_t c0, c1, x0, x1;
};

__device__ __forceinline__ Window window_of(const Levels& a, uint32_t g, uint32_t h, uint32_t p0,
                                            uint32_t p1) {
  Window w;
  w.c0 = search_le(a.ptr1, 0, g - 1, p0);
  w.c1 = search_le(a.ptr1, w.c0, g - 1, p1);
  w.x0 = search_le(a.ptr2, 0, h - 1, w.c0);
  w.x1 = search_le(a.ptr2, w.x0, h - 1, w.c1);
  return w;
}

// window_of by one whole warp (warp_search_le for each of the four bounds).
__device__ __forceinline__ Window warp_window_of(const Levels& a, uint32_t g, uint32_t h,
                                                 uint32_t p0, uint32_t p1) {
  Window w;
  w.c0 = warp_search_le(a.ptr1, 0, g - 1, p0);
  w.c1 = warp_search_le(a.ptr1, w.c0, g - 1, p1);
  w.x0 = warp_search_le(a.ptr2, 0, h - 1, w.c0);
  w.x1 = warp_search_le(a.ptr2, w.x0, h - 1, w.c1);
  return w;
}

// (x, y, z) of the point at position p inside a window that contains it.
__device__ __forceinline__ void point_at(const Levels& a, const Window& w, uint32_t p,
                                         uint32_t& x, uint32_t& y, uint32_t& z) {
  const uint32_t c = search_le(a.ptr1, w.c0, w.c1, p);
  const uint32_t xr = search_le(a.ptr2, w.x0, w.x1, c);
  x = __ldg(a.idx2 + xr);
  y = __ldg(a.idx1 + c);
  z = __ldg(a.idx0 + p);
}

// In-place inclusive max-scan of v[0, n) (n <= kThreads * CH) by a block of
// kThreads threads, each owning CH consecutive entries.  s_warp: kWarps
// words.  Contains two barriers.
template <int CH>
__device__ __forceinline__ void block_max_scan_u16(uint16_t* v, uint32_t n, uint32_t* s_warp) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t b0 = tid * CH;
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    if (b0 + i < n) m = max(m, (uint32_t)v[b0 + i]);
  }
  uint32_t inc = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= (uint32_t)o) inc = max(inc, t);
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  uint32_t run = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) run = 0;
  for (uint32_t i = 0; i < w; ++i) run = max(run, s_warp[i]);
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    if (b0 + i < n) {
      run = max(run, (uint32_t)v[b0 + i]);
      v[b0 + i] = (uint16_t)run;
    }
  }
  __syncthreads();
}

// Column and slab of every position of the window [p0, p0 + cnt) of a
// 3-level CGA (cnt <= kTile), relative to w.c0 and w.x0, in shared memory:
// each column start and slab start inside the window is written at its first
// position, then an inclusive max-scan carries it over the positions that
// follow.  col_of: cnt entries; slab_of: w.c1 - w.c0 + 1 entries (indexed by
// relative column).  All threads of the kThreads block must call it.
__device__ __forceinline__ void expand_window(const Levels& a, const Window& w, uint32_t p0,
                                              uint32_t cnt, uint16_t* col_of, uint16_t* slab_of,
                                              uint32_t* s_warp) {
  const uint32_t tid = threadIdx.x;
  const uint32_t ncol = w.c1 - w.c0 + 1;
  for (uint32_t j = tid; j < cnt; j += kThreads) col_of[j] = 0;
  for (uint32_t j = tid; j < ncol; j += kThreads) slab_of[j] = 0;
  __syncthreads();
  for (uint32_t c = w.c0 + 1 + tid; c <= w.c1; c += kThreads) {
    col_of[__ldg(a.ptr1 + c) - p0] = (uint16_t)(c - w.c0);
  }
  for (uint32_t x = w.x0 + 1 + tid; x <= w.x1; x += kThreads) {
    slab_of[__ldg(a.ptr2 + x) - w.c0] = (uint16_t)(x - w.x0);
  }
  __syncthreads();
  block_max_scan_u16<kTile / kThreads>(col_of, cnt, s_warp);
  block_max_scan_u16<kTile / kThreads>(slab_of, ncol, s_warp);
}

}  // namespace libcga
