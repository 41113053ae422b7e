// Sort pipeline of the CGA build (and of the xz / yz projections):
//   k_seg_init     headers and empty-CGA sentinels
//   k_keys_hist    quantize (+ rigid transform) and encode each point, or
//                  re-key a CGA point for a projection; per-segment digit
//                  histograms of every radix pass in the same read
//   k_onesweep     one LSD radix pass: warp-level digit ranking, decoupled
//                  look-back over tiles for the global digit offsets, scatter
//   k_compact      dedupe + CGA compaction (k_compact.cuh)
// Every kernel works on a batch of segments (clouds); a tile never spans two
// segments and look-back chains stop at the segment's first tile.
#include <algorithm>
#include <mutex>

#include "k_compact.cuh"

namespace libcga {

namespace {

__device__ __forceinline__ int find_seg(const SortSeg* __restrict__ segs, int S, uint32_t t) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Element count of a segment: known on the host for a build, read from the
// source header for a projection (the source is built earlier in the stream).
__device__ __forceinline__ uint32_t seg_count(const SortSeg& s) {
  if (s.from_cga) return (uint32_t)s.src.hdr->cnt[0];
  return s.n_host;
}

__global__ void k_seg_init(const SortSeg* __restrict__ segs, int S) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const Levels& o = segs[s].out;
  o.hdr->cnt[0] = 0;
  o.hdr->cnt[1] = 0;
  o.hdr->cnt[2] = 0;
  o.hdr->err = segs[s].from_cga ? segs[s].src.hdr->err : 0u;
  o.ptr1[0] = 0;
  if (o.nlevels == 3) o.ptr2[0] = 0;
}

// Keys of the tiles [t0, t1) plus per-segment histograms of every pass
// (digits of RB bits).
template <typename K, int RB>
__global__ void __launch_bounds__(kThreads) k_keys_hist(const SortSeg* __restrict__ segs, int S,
                                                        uint32_t total_tiles,
                                                        uint32_t tiles_per_cta, K* keys0,
                                                        uint32_t* hist) {
  constexpr int R = 1 << RB;
  __shared__ uint32_t s_hist[kMaxPasses][R];
  __shared__ float s_pts[kThreads * 3];
  __shared__ Window s_win;
  __shared__ uint16_t s_col[kTile], s_slab[kTile];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_err;
  const int tid = threadIdx.x;
  const uint32_t t0 = blockIdx.x * tiles_per_cta;
  const uint32_t t1 = min(t0 + tiles_per_cta, total_tiles);
  if (t0 >= t1) return;
  for (int i = tid; i < kMaxPasses * R; i += kThreads) (&s_hist[0][0])[i] = 0;
  if (tid == 0) s_err = 0;
  __syncthreads();
  int cur = find_seg(segs, S, t0);
  auto flush = [&](int s) {
    __syncthreads();
    const uint32_t passes = segs[s].passes;
    for (int i = tid; i < kMaxPasses * R; i += kThreads) {
      const uint32_t v = (&s_hist[0][0])[i];
      if (v != 0 && (uint32_t)(i >> RB) < passes) {
        atomicAdd(hist + (size_t)s * kMaxPasses * R + i, v);
      }
      (&s_hist[0][0])[i] = 0;
    }
    if (tid == 0 && s_err) {
      atomicOr(&segs[s].out.hdr->err, s_err);
      s_err = 0;
    }
    __syncthreads();
  };
  for (uint32_t t = t0; t < t1; ++t) {
    const int s = find_seg(segs, S, t);
    if (s != cur) {
      flush(cur);
      cur = s;
    }
    const SortSeg& sg = segs[s];
    const uint32_t n = seg_count(sg);
    const uint32_t start = (t - sg.tile_base) * kTile;
    if (start >= n) continue;
    const uint32_t cnt = min((uint32_t)kTile, n - start);
    K* out = keys0 + sg.key_base + start;
    const uint32_t passes = sg.passes;
    const uint32_t b = sg.bits;
    if (!sg.from_cga) {
      const float* src = sg.xyz + (size_t)start * 3;
      for (uint32_t c0 = 0; c0 < cnt; c0 += kThreads) {
        const uint32_t m = min((uint32_t)kThreads, cnt - c0);
        __syncthreads();
        for (uint32_t i = tid; i < m * 3; i += kThreads) s_pts[i] = __ldg(src + (size_t)c0 * 3 + i);
        __syncthreads();
        if ((uint32_t)tid < m) {
          K key;
          if (!point_key<K>(s_pts[3 * tid], s_pts[3 * tid + 1], s_pts[3 * tid + 2],
                            sg.has_x != 0, sg.X, sg.scale, sg.off, b, key)) {
            atomicOr(&s_err, kErrNonfinite);
          }
          out[c0 + tid] = key;
          for (uint32_t p = 0; p < passes; ++p) {
            atomicAdd(&s_hist[p][(uint32_t)(key >> (sg.bit0 + p * RB)) & (R - 1)], 1u);
          }
        }
      }
    } else {
      // projection: decode the source point, keep two axes
      const Levels& a = sg.src;
      if (tid < 32) {
        const Window wv = warp_window_of(a, (uint32_t)a.hdr->cnt[1], (uint32_t)a.hdr->cnt[2],
                                         start, start + cnt - 1);
        if (tid == 0) s_win = wv;
      }
      __syncthreads();
      const Window win = s_win;
      expand_window(a, win, start, cnt, s_col, s_slab, s_warp);
      for (uint32_t e = tid; e < cnt; e += kThreads) {
        const uint32_t cr = s_col[e];
        const uint32_t x = __ldg(a.idx2 + win.x0 + s_slab[cr]);
        const uint32_t y = __ldg(a.idx1 + win.c0 + cr);
        const uint32_t z = __ldg(a.idx0 + start + e);
        K key;
        if (sg.plane == 3) {
          const uint32_t L = sg.shift;
          key = ((K)(x >> L) << (2 * b)) | ((K)(y >> L) << b) | (K)(z >> L);
        } else if (sg.plane == 4) {
          key = (K)tree_key(x, y, z, sg.shift);
        } else {
          uint32_t u = x, v = y;
          if (sg.plane == 1) { u = x; v = z; }
          if (sg.plane == 2) { u = y; v = z; }
          key = ((K)u << b) | (K)v;
        }
        out[e] = key;
        for (uint32_t p = 0; p < passes; ++p) {
          atomicAdd(&s_hist[p][(uint32_t)(key >> (sg.bit0 + p * RB)) & (R - 1)], 1u);
        }
      }
      __syncthreads();
    }
  }
  flush(cur);
}

// Exclusive scan across a block of TH threads (s_warp: TH/32 words).
template <int TH, typename T>
__device__ __forceinline__ T block_scan_th(T v, T& total, T* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  T before = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < TH / 32; ++i) {
    const T x = s_warp[i];
    if (i < w) before += x;
    tot += x;
  }
  __syncthreads();
  total = tot;
  return before + inc - v;
}

// Dynamic shared memory of one pass block: the tile's keys, per-warp digit
// counts (u16), per-digit offsets and the warp scan words.
template <typename K, int TH, int RB>
constexpr size_t onesweep_smem() {
  return (size_t)kTile * sizeof(K) + (size_t)(TH / 32) * (1 << RB) * 2 + (size_t)(1 << RB) * 4 +
         (size_t)(TH / 32) * 4;
}

// Blocks per SM a pass kernel is compiled for (its register budget), per
// threads per tile; measured on GB300 (30M-key builds): more resident warps
// hide more of the key loads and look-back waits than the few spilled values
// cost.
#ifndef CGA_SORT_BLOCKS_512
#define CGA_SORT_BLOCKS_512 4
#endif
#ifndef CGA_SORT_BLOCKS_256
#define CGA_SORT_BLOCKS_256 5
#endif

// One LSD pass over digit `pass` (RB bits) of every segment that still needs
// it.  A tile of kTile keys is TH threads x kTile/TH keys (warp-striped);
// threads tid < 2^RB own one digit each for the per-digit steps.
template <typename K, int TH, int RB>
__global__ void __launch_bounds__(TH, TH == 512 ? CGA_SORT_BLOCKS_512 : CGA_SORT_BLOCKS_256) k_onesweep(const SortSeg* __restrict__ segs, int S,
                                                 int pass, const K* __restrict__ in,
                                                 K* __restrict__ out,
                                                 const uint32_t* __restrict__ hist,
                                                 uint32_t* look, uint32_t* counter) {
  constexpr int IT = kTile / TH, WARPS = TH / 32, R = 1 << RB;
  static_assert(IT * TH == kTile && TH >= R, "tile shape");
  extern __shared__ __align__(16) unsigned char s_raw[];
  K* s_keys = reinterpret_cast<K*>(s_raw);
  uint16_t (*s_wh)[R] = reinterpret_cast<uint16_t (*)[R]>(s_raw + (size_t)kTile * sizeof(K));
  uint32_t* s_off = reinterpret_cast<uint32_t*>(s_raw + (size_t)kTile * sizeof(K) +
                                                (size_t)WARPS * R * 2);
  uint32_t* s_scan = s_off + R;
  __shared__ uint32_t s_tile;
  __shared__ int s_seg;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    const uint32_t t = atomicAdd(counter, 1u);
    s_tile = t;
    s_seg = find_seg(segs, S, t);
  }
  for (int i = tid; i < WARPS * R; i += TH) (&s_wh[0][0])[i] = 0;
  __syncthreads();
  const uint32_t t = s_tile;
  const int s = s_seg;
  const SortSeg& sg = segs[s];
  if (pass >= (int)sg.passes) return;
  const uint32_t n = seg_count(sg);
  const uint32_t lt = t - sg.tile_base;
  const uint32_t start = lt * kTile;
  if (start >= n) return;
  const uint32_t cnt = min((uint32_t)kTile, n - start);
  const K* src = in + sg.key_base + start;
  const int shift = (int)sg.bit0 + pass * RB;

  K k[IT];
  uint32_t dg[IT], rk[IT];
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const uint32_t e = (uint32_t)(w * 32 * IT + i * 32 + lane);
    const bool v = e < cnt;
    k[i] = v ? src[e] : (K)0;
    dg[i] = v ? ((uint32_t)(k[i] >> shift) & (R - 1)) : 0xffffffffu;
  }
  // warp-level ranking: lanes holding the same digit form one peer group
  uint16_t* wh = s_wh[w];
  const uint32_t ltm = lanemask_lt();
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const uint32_t d = dg[i];
    // lanes with the same digit: one warp vote per digit bit and one for
    // validity (votes issue faster than a match over the digit)
    uint32_t peers = __ballot_sync(0xffffffffu, d < (uint32_t)R);
    if (d >= (uint32_t)R) peers = ~peers;
#pragma unroll
    for (int bit = 0; bit < RB; ++bit) {
      const uint32_t v = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
      peers &= ((d >> bit) & 1u) ? v : ~v;
    }
    const uint32_t base = (d < (uint32_t)R) ? wh[d] : 0u;
    __syncwarp();
    if (d < (uint32_t)R && lane == __ffs(peers) - 1) wh[d] = (uint16_t)(base + __popc(peers));
    __syncwarp();
    rk[i] = base + __popc(peers & ltm);
  }
  __syncthreads();
  // per digit (thread tid == digit): warp offsets, tile count, publish
  const int d = tid;
  const bool owner = tid < R;
  uint32_t tile_cnt = 0;
  uint32_t* my = look + (size_t)t * R + d;
  if (owner) {
    for (int x = 0; x < WARPS; ++x) {
      const uint32_t v = s_wh[x][d];
      s_wh[x][d] = (uint16_t)tile_cnt;
      tile_cnt += v;
    }
    st_relaxed(my, (lt == 0 ? kFlagInc : kFlagAgg) | tile_cnt);
  }
  uint32_t tot;
  const uint32_t bin_start = block_scan_th<TH>(owner ? tile_cnt : 0u, tot, s_scan);
  const uint32_t hv = owner ? hist[((size_t)s * kMaxPasses + pass) * R + d] : 0u;
  const uint32_t dbase = block_scan_th<TH>(hv, tot, s_scan);
  if (owner) s_off[d] = bin_start;
  __syncthreads();
  bool bad = false;
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    if (dg[i] < (uint32_t)R) {
      const uint32_t pos = s_off[dg[i]] + s_wh[w][dg[i]] + rk[i];
      if (pos < (uint32_t)kTile) s_keys[pos] = k[i]; else bad = true;
    }
  }
  uint32_t excl = 0;
  if (owner && lt > 0) {
    excl = lookback(look + d, R, t, sg.tile_base, &sg.out.hdr->err);
    st_relaxed(my, kFlagInc | ((excl + tile_cnt) & kValMask));
  }
  __syncthreads();
  if (owner) s_off[d] = dbase + excl - bin_start;
  __syncthreads();
  K* dst = out + sg.key_base;
  for (uint32_t e = tid; e < cnt; e += TH) {
    const K key = s_keys[e];
    const uint32_t pos = s_off[(uint32_t)(key >> shift) & (R - 1)] + e;
    if (pos < n) dst[pos] = key; else bad = true;
  }
  if (bad) atomicOr(&sg.out.hdr->err, kErrInternal);
}


template <typename K, int LEVELS>
__global__ void __launch_bounds__(kThreads) k_compact(const SortSeg* __restrict__ segs, int S,
                                                      const K* __restrict__ keys0,
                                                      const K* __restrict__ keys1,
                                                      uint32_t* clook, uint32_t* counter) {
  __shared__ CompactSmem sm;
  __shared__ uint32_t s_tile;
  __shared__ int s_seg;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    const uint32_t t = atomicAdd(counter, 1u);
    s_tile = t;
    s_seg = find_seg(segs, S, t);
  }
  __syncthreads();
  const uint32_t t = s_tile;
  const SortSeg& sg = segs[s_seg];
  const uint32_t n = seg_count(sg);
  const uint32_t lt = t - sg.tile_base;
  const uint32_t start = lt * kTile;
  if (start >= n) return;
  const uint32_t cnt = min((uint32_t)kTile, n - start);
  const K* src = ((sg.passes & 1u) ? keys1 : keys0) + sg.key_base + start;
  K k[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t e = (uint32_t)(w * 32 * kItems + i * 32 + lane);
    k[i] = (e < cnt) ? src[e] : (K)0;
  }
  const bool has_prev = start > 0;
  const K prev = has_prev ? src[-1] : (K)0;
  const bool last = (start + cnt == n);
  compact_tile<LEVELS, K>(k, cnt, has_prev, prev, t, sg.tile_base, last, sg.out, clook, sm);
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

size_t sort_scratch_bytes(uint64_t total_keys, uint32_t total_tiles, int S, bool key64,
                          uint32_t radix_bits) {
  const size_t ks = key64 ? 8 : 4;
  const size_t R = (size_t)1 << radix_bits;
  size_t b = 0;
  b += align_up(total_keys * ks) * 2;
  b += align_up((size_t)S * kMaxPasses * R * 4);
  b += align_up((size_t)kMaxPasses * total_tiles * R * 4);
  b += align_up((size_t)total_tiles * 3 * 4);
  b += align_up((kMaxPasses + 1) * 4);
  b += align_up((size_t)S * sizeof(SortSeg));
  return b;
}

SortScratch sort_scratch_carve(void* base, uint64_t total_keys, uint32_t total_tiles, int S,
                               bool key64, const Tuning& tu) {
  const size_t ks = key64 ? 8 : 4;
  const size_t R = (size_t)1 << tu.radix_bits;
  char* p = static_cast<char*>(base);
  SortScratch sc{};
  sc.radix_bits = tu.radix_bits;
  sc.sort_threads = tu.sort_threads;
  sc.keys0 = p;
  p += align_up(total_keys * ks);
  sc.keys1 = p;
  p += align_up(total_keys * ks);
  char* z0 = p;
  sc.hist = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)S * kMaxPasses * R * 4);
  sc.look = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)kMaxPasses * total_tiles * R * 4);
  sc.clook = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)total_tiles * 3 * 4);
  sc.counters = reinterpret_cast<uint32_t*>(p);
  p += align_up((kMaxPasses + 1) * 4);
  sc.zero_bytes = (size_t)(p - z0);
  sc.segs = reinterpret_cast<SortSeg*>(p);
  return sc;
}

int device_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <typename K, int TH, int RB>
static cudaError_t set_pass_smem() {
  return cudaFuncSetAttribute(k_onesweep<K, TH, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)onesweep_smem<K, TH, RB>());
}

template <typename K, int TH, int RB>
static void launch_shape(int S, uint32_t total_tiles, uint32_t max_passes, const SortScratch& sc,
                         cudaStream_t stream) {
  K* k0 = static_cast<K*>(sc.keys0);
  K* k1 = static_cast<K*>(sc.keys1);
  constexpr size_t smem = onesweep_smem<K, TH, RB>();
  for (uint32_t p = 0; p < max_passes; ++p) {
    const K* in = (p & 1) ? k1 : k0;
    K* out = (p & 1) ? k0 : k1;
    k_onesweep<K, TH, RB><<<total_tiles, TH, smem, stream>>>(
        sc.segs, S, (int)p, in, out, sc.hist, sc.look + ((size_t)p * total_tiles << RB),
        sc.counters + p);
  }
  count_launch(max_passes);
}

template <typename K>
static void launch_passes(int S, uint32_t total_tiles, uint32_t max_passes, const SortScratch& sc,
                          cudaStream_t stream) {
  if (sc.radix_bits == 9) {
    launch_shape<K, 512, 9>(S, total_tiles, max_passes, sc, stream);
  } else if (sc.sort_threads == 256) {
    launch_shape<K, 256, 8>(S, total_tiles, max_passes, sc, stream);
  } else {
    launch_shape<K, 512, 8>(S, total_tiles, max_passes, sc, stream);
  }
}

cudaError_t init_sort_kernels() {
  static std::once_flag once;
  static cudaError_t rc = cudaSuccess;
  std::call_once(once, [] {
    const cudaError_t es[] = {
        set_pass_smem<uint32_t, 256, 8>(),           set_pass_smem<uint32_t, 512, 8>(),
        set_pass_smem<uint32_t, 512, 9>(),           set_pass_smem<unsigned long long, 256, 8>(),
        set_pass_smem<unsigned long long, 512, 8>(), set_pass_smem<unsigned long long, 512, 9>()};
    for (cudaError_t e : es) {
      if (e != cudaSuccess && rc == cudaSuccess) rc = e;
    }
  });
  return rc;
}

cudaError_t run_radix_passes(int S, uint32_t total_tiles, uint32_t max_passes, bool key64,
                             const SortScratch& sc, cudaStream_t stream) {
  if (total_tiles == 0) return cudaSuccess;
  const cudaError_t ei = init_sort_kernels();
  if (ei != cudaSuccess) return ei;
  if (key64) {
    launch_passes<unsigned long long>(S, total_tiles, max_passes, sc, stream);
  } else {
    launch_passes<uint32_t>(S, total_tiles, max_passes, sc, stream);
  }
  return cudaGetLastError();
}

template <typename K>
static cudaError_t launch_pipeline(int S, uint32_t total_tiles, uint32_t max_passes, int levels,
                                   const SortScratch& sc, cudaStream_t stream) {
  K* k0 = static_cast<K*>(sc.keys0);
  K* k1 = static_cast<K*>(sc.keys1);
  const uint32_t ctas = std::min<uint32_t>(total_tiles, (uint32_t)device_sm_count() * 4);
  const uint32_t per = (total_tiles + ctas - 1) / ctas;
  const cudaError_t ei = init_sort_kernels();
  if (ei != cudaSuccess) return ei;
  if (sc.radix_bits == 9) {
    k_keys_hist<K, 9><<<ctas, kThreads, 0, stream>>>(sc.segs, S, total_tiles, per, k0, sc.hist);
  } else {
    k_keys_hist<K, 8><<<ctas, kThreads, 0, stream>>>(sc.segs, S, total_tiles, per, k0, sc.hist);
  }
  count_launch(2);
  launch_passes<K>(S, total_tiles, max_passes, sc, stream);
  if (levels == 3) {
    k_compact<K, 3><<<total_tiles, kThreads, 0, stream>>>(sc.segs, S, k0, k1, sc.clook,
                                                          sc.counters + kMaxPasses);
  } else {
    k_compact<K, 2><<<total_tiles, kThreads, 0, stream>>>(sc.segs, S, k0, k1, sc.clook,
                                                          sc.counters + kMaxPasses);
  }
  return cudaGetLastError();
}

template <typename K>
static void launch_keys(int S, uint32_t total_tiles, const SortScratch& sc, cudaStream_t stream) {
  const uint32_t ctas = std::min<uint32_t>(total_tiles, (uint32_t)device_sm_count() * 4);
  const uint32_t per = (total_tiles + ctas - 1) / ctas;
  K* k0 = static_cast<K*>(sc.keys0);
  if (sc.radix_bits == 9) {
    k_keys_hist<K, 9><<<ctas, kThreads, 0, stream>>>(sc.segs, S, total_tiles, per, k0, sc.hist);
  } else {
    k_keys_hist<K, 8><<<ctas, kThreads, 0, stream>>>(sc.segs, S, total_tiles, per, k0, sc.hist);
  }
  count_launch(1);
}

cudaError_t run_sort_keys_device(int S, uint32_t total_tiles, uint32_t max_passes,
                                 const SortScratch& sc, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(sc.hist, 0, sc.zero_bytes, stream);
  if (e != cudaSuccess || total_tiles == 0) return e;
  e = init_sort_kernels();
  if (e != cudaSuccess) return e;
  launch_keys<unsigned long long>(S, total_tiles, sc, stream);
  launch_passes<unsigned long long>(S, total_tiles, max_passes, sc, stream);
  return cudaGetLastError();
}

cudaError_t run_sort_device(int S, uint32_t total_tiles, uint32_t max_passes, bool key64,
                            int levels, const SortScratch& sc, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(sc.hist, 0, sc.zero_bytes, stream);
  if (e != cudaSuccess) return e;
  k_seg_init<<<(S + 127) / 128, 128, 0, stream>>>(sc.segs, S);
  count_launch(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || total_tiles == 0) return e;
  return key64 ? launch_pipeline<unsigned long long>(S, total_tiles, max_passes, levels, sc, stream)
               : launch_pipeline<uint32_t>(S, total_tiles, max_passes, levels, sc, stream);
}

size_t wait_selftest_bytes() {
  return align_up(sizeof(Header)) + sort_scratch_bytes(2 * kTile, 2, 1, true);
}

// One radix-pass tile that draws tile id 1 of a two-tile segment whose tile 0
// never runs: its look-back word for tile 0 is never published, so the wait
// must give up on its own and record kErrTimeout in *hdr.
cudaError_t run_wait_selftest(void* scratch, cudaStream_t stream) {
  const size_t bytes = wait_selftest_bytes();
  Header* hdr = static_cast<Header*>(scratch);
  const SortScratch sc = sort_scratch_carve(static_cast<char*>(scratch) + align_up(sizeof(Header)),
                                            2 * kTile, 2, 1, true);
  SortSeg seg{};
  seg.n_host = 2 * kTile;
  seg.passes = 1;
  seg.num_tiles = 2;
  seg.out.hdr = hdr;
  const uint32_t first_id = 1;
  cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc.segs, &seg, sizeof(SortSeg), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(sc.counters, &first_id, sizeof(uint32_t), cudaMemcpyHostToDevice, stream);
  }
  if (e != cudaSuccess) return e;
  e = init_sort_kernels();
  if (e != cudaSuccess) return e;
  k_onesweep<unsigned long long, 512, 8>
      <<<1, 512, onesweep_smem<unsigned long long, 512, 8>(), stream>>>(
      sc.segs, 1, 0, static_cast<const unsigned long long*>(sc.keys0),
      static_cast<unsigned long long*>(sc.keys1), sc.hist, sc.look, sc.counters);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_sort_pipeline(const SortSeg* h_segs, int S, uint32_t total_tiles,
                              uint32_t max_passes, bool key64, const SortScratch& sc,
                              cudaStream_t stream) {
  cudaError_t e = cudaMemcpyAsync(sc.segs, h_segs, sizeof(SortSeg) * S, cudaMemcpyHostToDevice,
                                  stream);
  if (e != cudaSuccess) return e;
  return run_sort_device(S, total_tiles, max_passes, key64, (int)h_segs[0].out.nlevels, sc,
                         stream);
}

}  // namespace libcga
