// Operations on built CGAs: decode, merge, xy projection, exact NN search.
#include <algorithm>

#include "k_compact.cuh"

namespace libcga {

namespace {

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ decode
// Lossless inverse of the build: the walk X -> Y -> Z of Sec. V-A, done per
// tile of Z positions (the tile's window is expanded into per-position column
// and slab indices in shared memory).
__global__ void __launch_bounds__(kThreads) k_decode(Levels a, uint32_t* __restrict__ xyz) {
  __shared__ Window s_win;
  __shared__ uint16_t s_col[kTile], s_slab[kTile];
  __shared__ uint32_t s_warp[kWarps];
  const uint32_t u = (uint32_t)a.hdr->cnt[0];
  const uint32_t start = blockIdx.x * kTile;
  if (start >= u) return;
  const uint32_t cnt = min((uint32_t)kTile, u - start);
  if (threadIdx.x < 32) {
    const Window wv =
        warp_window_of(a, (uint32_t)a.hdr->cnt[1], (uint32_t)a.hdr->cnt[2], start, start + cnt - 1);
    if (threadIdx.x == 0) s_win = wv;
  }
  __syncthreads();
  const Window w = s_win;
  expand_window(a, w, start, cnt, s_col, s_slab, s_warp);
  for (uint32_t e = threadIdx.x; e < cnt; e += kThreads) {
    const uint32_t cr = s_col[e];
    uint32_t* o = xyz + (size_t)(start + e) * 3;
    o[0] = __ldg(a.idx2 + w.x0 + s_slab[cr]);
    o[1] = __ldg(a.idx1 + w.c0 + cr);
    o[2] = __ldg(a.idx0 + start + e);
  }
}

// ------------------------------------------------------------------- merge
__device__ __forceinline__ int find_pair_spl(const MergePair* __restrict__ P, int S, uint32_t i) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P[mid].spl_base <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_pair_tile(const MergePair* __restrict__ P, int S, uint32_t t) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t n_splitters(uint32_t u, uint32_t reserved, uint32_t half) {
  const uint32_t k = u > 0 ? (u - 1) / half : 0u;
  return min(k, reserved);
}

// Output header, empty-CGA sentinels, first and last tile bounds.
__global__ void k_merge_init(const MergePair* __restrict__ pairs, int S, uint32_t half,
                             uint32_t* bounds, uint32_t* ntiles) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S) return;
  const MergePair& P = pairs[p];
  const uint32_t uA = (uint32_t)P.a.hdr->cnt[0], uB = (uint32_t)P.b.hdr->cnt[0];
  const uint32_t NA = n_splitters(uA, P.spl_a, half), NB = n_splitters(uB, P.spl_b, half);
  const uint32_t nt = NA + NB + 1;
  ntiles[p] = nt;
  uint32_t* bnd = bounds + 2 * ((size_t)P.tile_base + p);
  bnd[0] = 0;
  bnd[1] = 0;
  bnd[2 * nt] = uA;
  bnd[2 * nt + 1] = uB;
  P.out.hdr->cnt[0] = 0;
  P.out.hdr->cnt[1] = 0;
  P.out.hdr->cnt[2] = 0;
  P.out.hdr->err = P.a.hdr->err | P.b.hdr->err;
  P.out.ptr1[0] = 0;
  P.out.ptr2[0] = 0;
}

// Tile cuts, one warp per splitter.  Splitter k of A is A's key s at
// position (k + 1) * half; its cut is (rank_A(s), rank_B(s)) = ((k + 1) *
// half, #B keys < s), and its place among all splitters (A's before B's on
// equal keys) is k + #B splitters < s, where B splitter j (the key at
// (j + 1) * half) is below s exactly when (j + 1) * half < rank_B(s).  B's
// splitters mirror this with #A keys <= s.  The Sec. V-A lookup gives the
// ranks.
__global__ void k_merge_cuts(const MergePair* __restrict__ pairs, int S, uint32_t total,
                             uint32_t half, uint32_t* bounds) {
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (i >= total) return;
  const int p = find_pair_spl(pairs, S, i);
  const MergePair& P = pairs[p];
  const uint32_t local = i - P.spl_base;
  const uint32_t uA = (uint32_t)P.a.hdr->cnt[0], uB = (uint32_t)P.b.hdr->cnt[0];
  const uint32_t NA = n_splitters(uA, P.spl_a, half), NB = n_splitters(uB, P.spl_b, half);
  const bool isA = local < P.spl_a;
  const uint32_t k = isA ? local : local - P.spl_a;
  if (k >= (isA ? NA : NB)) return;
  const Levels& own = isA ? P.a : P.b;
  const Levels& oth = isA ? P.b : P.a;
  const unsigned long long s =
      warp_key_at(own, (uint32_t)own.hdr->cnt[1], (uint32_t)own.hdr->cnt[2], (k + 1) * half);
  bool found = false;
  const uint32_t r = warp_rank_of(oth, (uint32_t)oth.hdr->cnt[2], s, &found);
  // other-side splitters before this one: below s (A's turn), or at most s (B's)
  const uint32_t rk = isA ? r : r + (found ? 1u : 0u);
  const uint32_t before = rk > 0 ? min(isA ? NB : NA, (rk - 1) / half) : 0u;
  const uint32_t pos = k + before;
  if (lane == 0) {
    uint32_t* bnd = bounds + 2 * ((size_t)P.tile_base + p);
    bnd[2 * (pos + 1)] = isA ? (k + 1) * half : r;
    bnd[2 * (pos + 1) + 1] = isA ? r : (k + 1) * half;
  }
}

// Merge one tile: decode both runs (at most MH points each) into shared
// memory, merge-path split per thread, sequential merge, then the shared
// dedupe + compaction.
template <int MH>
__global__ void __launch_bounds__(kThreads) k_merge_tiles(const MergePair* __restrict__ pairs,
                                                          int S, const uint32_t* __restrict__ bounds,
                                                          const uint32_t* __restrict__ ntiles,
                                                          uint32_t* clook, uint32_t* counter) {
  constexpr int IT = 2 * MH / kThreads;  // merged keys per thread
  static_assert(IT * kThreads == 2 * MH && 2 * MH <= kTile, "merge tile shape");
  __shared__ unsigned long long s_ab[2 * MH];
  __shared__ uint16_t s_col[MH], s_slab[MH];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ CompactSmem sm;
  __shared__ Window s_wa, s_wb;
  __shared__ unsigned long long s_prev, s_prev2[2];
  __shared__ uint32_t s_tile, s_has_prev;
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    const uint32_t t = atomicAdd(counter, 1u);
    s_tile = t;
    s_p = find_pair_tile(pairs, S, t);
  }
  __syncthreads();
  const uint32_t t = s_tile;
  const int p = s_p;
  const MergePair& P = pairs[p];
  const uint32_t lt = t - P.tile_base;
  const uint32_t nt = ntiles[p];
  if (lt >= nt) return;
  const uint32_t* bnd = bounds + 2 * ((size_t)P.tile_base + p + lt);
  uint32_t a0 = bnd[0], b0 = bnd[1], a1 = bnd[2], b1 = bnd[3];
  uint32_t na = a1 - a0, nb = b1 - b0;
  const bool bad = a1 < a0 || b1 < b0 || na > (uint32_t)MH || nb > (uint32_t)MH;
  if (bad) {
    na = 0;
    nb = 0;
  }
  const uint32_t gA = (uint32_t)P.a.hdr->cnt[1], hA = (uint32_t)P.a.hdr->cnt[2];
  const uint32_t gB = (uint32_t)P.b.hdr->cnt[1], hB = (uint32_t)P.b.hdr->cnt[2];
  // the tile's windows in both inputs and the key just before it: four
  // independent warp-cooperative searches
  if (w == 0) {
    if (bad && lane == 0) atomicOr(&P.out.hdr->err, kErrInternal);
    if (na) {
      const Window wa = warp_window_of(P.a, gA, hA, a0, a1 - 1);
      if (lane == 0) s_wa = wa;
    }
  } else if (w == 1) {
    if (nb) {
      const Window wb = warp_window_of(P.b, gB, hB, b0, b1 - 1);
      if (lane == 0) s_wb = wb;
    }
  } else if (w == 2) {
    const unsigned long long ka = a0 > 0 ? warp_key_at(P.a, gA, hA, a0 - 1) : 0ull;
    if (lane == 0) s_prev2[0] = ka;
  } else if (w == 3) {
    const unsigned long long kb = b0 > 0 ? warp_key_at(P.b, gB, hB, b0 - 1) : 0ull;
    if (lane == 0) s_prev2[1] = kb;
  }
  __syncthreads();
  if (tid == 0) {
    // the predecessor key of the merged run is the larger of the two
    s_prev = max(a0 > 0 ? s_prev2[0] : 0ull, b0 > 0 ? s_prev2[1] : 0ull);
    s_has_prev = (a0 > 0 || b0 > 0) ? 1u : 0u;
  }
  __syncthreads();
  const uint32_t bA = P.a.bits;
  // decode both runs (tile-uniform branches: the window expansion has barriers)
  if (na) {
    const Window wa = s_wa;
    expand_window(P.a, wa, a0, na, s_col, s_slab, s_warp);
    for (uint32_t e = tid; e < na; e += kThreads) {
      const uint32_t cr = s_col[e];
      const uint32_t x = __ldg(P.a.idx2 + wa.x0 + s_slab[cr]), y = __ldg(P.a.idx1 + wa.c0 + cr);
      s_ab[e] = ((unsigned long long)x << (2 * bA)) | ((unsigned long long)y << bA) |
                __ldg(P.a.idx0 + a0 + e);
    }
    __syncthreads();
  }
  if (nb) {
    const Window wb = s_wb;
    expand_window(P.b, wb, b0, nb, s_col, s_slab, s_warp);
    for (uint32_t e = tid; e < nb; e += kThreads) {
      const uint32_t cr = s_col[e];
      const uint32_t x = __ldg(P.b.idx2 + wb.x0 + s_slab[cr]), y = __ldg(P.b.idx1 + wb.c0 + cr);
      s_ab[MH + e] = ((unsigned long long)x << (2 * bA)) | ((unsigned long long)y << bA) |
                     __ldg(P.b.idx0 + b0 + e);
    }
  }
  __syncthreads();
  const uint32_t cnt = na + nb;
  const uint32_t diag = min((uint32_t)(tid * IT), cnt);
  uint32_t lo = diag > nb ? diag - nb : 0u, hi = min(diag, na);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s_ab[mid] <= s_ab[MH + diag - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  uint32_t i = lo, j = diag - lo;
  unsigned long long r[IT];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const bool takeA = i < na && (j >= nb || s_ab[i] <= s_ab[MH + j]);
    const bool any = i < na || j < nb;
    unsigned long long v = 0;
    if (any) v = takeA ? s_ab[i] : s_ab[MH + j];
    if (any) {
      if (takeA) ++i; else ++j;
    }
    r[it] = v;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint32_t pos = diag + it;
    if (pos < cnt) s_ab[pos] = r[it];
  }
  __syncthreads();
  unsigned long long k[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const uint32_t e = (uint32_t)(w * 32 * kItems + it * 32 + lane);
    k[it] = (e < cnt) ? s_ab[e] : 0ull;
  }
  compact_tile<3, unsigned long long>(k, cnt, s_has_prev != 0, s_prev, t, P.tile_base,
                                      lt == nt - 1, P.out, clook, sm);
}

// ------------------------------------------------------- coarse slab index
__global__ void k_coarse_slab_index(Levels a, Levels c, uint32_t shift, uint32_t* xs) {
  const uint32_t hc = (uint32_t)c.hdr->cnt[2], ha = (uint32_t)a.hdr->cnt[2];
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= hc; k += stride) {
    xs[k] = (k == hc) ? ha : lower_bound_u16(a.idx2, 0, ha, (uint32_t)__ldg(c.idx2 + k) << shift);
  }
}

// ---------------------------------------------------------- child columns
// Where each coarse column's cell starts in every finer slab below it: the
// refinement of a cell reads its starting columns instead of searching.
__global__ void k_child_columns(Levels f, Levels c, const uint32_t* __restrict__ xs, uint32_t dsh,
                                uint32_t* child) {
  const uint32_t gc = (uint32_t)c.hdr->cnt[1], hc = (uint32_t)c.hdr->cnt[2];
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t col = blockIdx.x * blockDim.x + threadIdx.x; col < gc; col += stride) {
    const uint32_t X = search_le(c.ptr2, 0, hc - 1, col);
    const uint32_t fx0 = __ldg(xs + X), fx1 = __ldg(xs + X + 1);
    const uint32_t ylo = (uint32_t)__ldg(c.idx1 + col) << dsh;
    for (uint32_t j = 0; j < fx1 - fx0; ++j) {
      const uint32_t xi = fx0 + j;
      child[((size_t)col << dsh) + j] =
          lower_bound_u16(f.idx1, __ldg(f.ptr2 + xi), __ldg(f.ptr2 + xi + 1), ylo);
    }
  }
}

// -------------------------------------------------------- column table
// The column table of the NN search (the CGA's, and each coarse level's):
// per column its first voxel, its end and its z range (lowest | highest <<
// 16), read by one 16-byte load; the z range settles a column without a
// search when the query lies below or above all of it.
__global__ void k_column_table(Levels a, uint4* t) {
  const uint32_t g = (uint32_t)a.hdr->cnt[1];
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < g; c += stride) {
    const uint32_t zs = __ldg(a.ptr1 + c), ze = __ldg(a.ptr1 + c + 1);
    t[c] = make_uint4(zs, ze,
                      (uint32_t)__ldg(a.idx0 + zs) | ((uint32_t)__ldg(a.idx0 + ze - 1) << 16), 0u);
  }
}

// ------------------------------------------------------------ x directory
// The dense per-x-value table of G-Arrays (Sec. V), here only as a lookup
// accelerator: xdir[v] = number of stored x values below v.
__global__ void k_x_directory(Levels a, uint32_t* xdir) {
  const uint32_t h = (uint32_t)a.hdr->cnt[2];
  const uint32_t n = 1u << a.bits;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
    xdir[v] = lower_bound_u16(a.idx2, 0, h, v);
  }
}

// ------------------------------------------------------------- projection xy
__device__ __forceinline__ void project_xy_body(const Levels& a, const Levels& o, uint32_t t,
                                                uint32_t stride) {
  const uint32_t g = (uint32_t)a.hdr->cnt[1], h = (uint32_t)a.hdr->cnt[2];
  for (uint32_t i = t; i < g; i += stride) o.idx0[i] = a.idx1[i];
  for (uint32_t i = t; i < h; i += stride) o.idx1[i] = a.idx2[i];
  for (uint32_t i = t; i <= h; i += stride) o.ptr1[i] = a.ptr2[i];
  if (t == 0) {
    o.hdr->cnt[0] = g;
    o.hdr->cnt[1] = h;
    o.hdr->cnt[2] = 0;
    o.hdr->err = a.hdr->err;
  }
}

// One projection per blockIdx.y.
__global__ void k_project_xy_batch(const ProjPair* __restrict__ pairs) {
  const ProjPair& P = pairs[blockIdx.y];
  project_xy_body(P.a, P.out, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// The xy projection of a CGA is its top two levels (X_index, X_pointer,
// Y_index): copy them.
__global__ void k_project_xy(Levels a, Levels o) {
  project_xy_body(a, o, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

}  // namespace

cudaError_t run_decode(const Levels& a, uint32_t* xyz, cudaStream_t stream) {
  const uint64_t tiles = (a.cap + kTile - 1) / kTile;
  if (tiles == 0) return cudaSuccess;
  k_decode<<<(unsigned)tiles, kThreads, 0, stream>>>(a, xyz);
  count_launch(1);
  return cudaGetLastError();
}

size_t merge_scratch_bytes(uint32_t total_spl, uint32_t total_tiles, int S) {
  (void)total_spl;
  size_t b = 0;
  b += align_up(((size_t)total_tiles + S) * 2 * 4 + 8);
  b += align_up((size_t)S * 4);
  b += align_up((size_t)total_tiles * 3 * 4);
  b += align_up(4);
  b += align_up((size_t)S * sizeof(MergePair));
  return b;
}

MergeScratch merge_scratch_carve(void* base, uint32_t total_spl, uint32_t total_tiles, int S,
                                 uint32_t half) {
  char* p = static_cast<char*>(base);
  MergeScratch sc{};
  sc.half = half;
  (void)total_spl;
  sc.bounds = reinterpret_cast<uint32_t*>(p);
  p += align_up(((size_t)total_tiles + S) * 2 * 4 + 8);
  sc.ntiles = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)S * 4);
  char* z0 = p;
  sc.clook = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)total_tiles * 3 * 4);
  sc.counter = reinterpret_cast<uint32_t*>(p);
  p += align_up(4);
  sc.zero_bytes = (size_t)(p - z0);
  sc.pairs = reinterpret_cast<MergePair*>(p);
  return sc;
}

cudaError_t run_merge_device(int S, uint32_t total_spl, uint32_t total_tiles,
                             const MergeScratch& sc, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(sc.clook, 0, sc.zero_bytes, stream);
  if (e != cudaSuccess) return e;
  if (sc.half != 512 && sc.half != 1024 && sc.half != 2048) return cudaErrorInvalidValue;
  k_merge_init<<<(S + 127) / 128, 128, 0, stream>>>(sc.pairs, S, sc.half, sc.bounds, sc.ntiles);
  count_launch(total_spl > 0 ? 3 : 2);
  if (total_spl > 0) {
    k_merge_cuts<<<(total_spl + 7) / 8, 256, 0, stream>>>(sc.pairs, S, total_spl, sc.half,
                                                         sc.bounds);
  }
  if (sc.half == 512) {
    k_merge_tiles<512><<<total_tiles, kThreads, 0, stream>>>(sc.pairs, S, sc.bounds, sc.ntiles,
                                                             sc.clook, sc.counter);
  } else if (sc.half == 1024) {
    k_merge_tiles<1024><<<total_tiles, kThreads, 0, stream>>>(sc.pairs, S, sc.bounds, sc.ntiles,
                                                              sc.clook, sc.counter);
  } else {
    k_merge_tiles<2048><<<total_tiles, kThreads, 0, stream>>>(sc.pairs, S, sc.bounds, sc.ntiles,
                                                              sc.clook, sc.counter);
  }
  return cudaGetLastError();
}

cudaError_t run_merge(const MergePair* h_pairs, int S, uint32_t total_spl, uint32_t total_tiles,
                      const MergeScratch& sc, cudaStream_t stream) {
  cudaError_t e = cudaMemcpyAsync(sc.pairs, h_pairs, sizeof(MergePair) * S,
                                  cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return e;
  return run_merge_device(S, total_spl, total_tiles, sc, stream);
}

cudaError_t run_project_xy(const Levels& a, const Levels& out, cudaStream_t stream) {
  const uint64_t work = std::max<uint64_t>(a.cap1, 1);
  const unsigned blocks = (unsigned)std::min<uint64_t>((work + 255) / 256,
                                                       (uint64_t)device_sm_count() * 8);
  k_project_xy<<<blocks, 256, 0, stream>>>(a, out);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_coarse_slab_index(const Levels& a, const Levels& c, uint32_t shift, uint32_t* xs,
                                  cudaStream_t stream) {
  const uint64_t work = c.cap2 + 1;
  const unsigned blocks = (unsigned)std::min<uint64_t>((work + 255) / 256,
                                                       (uint64_t)device_sm_count() * 8);
  k_coarse_slab_index<<<blocks, 256, 0, stream>>>(a, c, shift, xs);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_child_columns(const Levels& f, const Levels& c, const uint32_t* xs, uint32_t dsh,
                              uint32_t* child, cudaStream_t stream) {
  const uint64_t work = std::max<uint64_t>(c.cap1, 1);
  const unsigned blocks = (unsigned)std::min<uint64_t>((work + 255) / 256,
                                                       (uint64_t)device_sm_count() * 8);
  k_child_columns<<<blocks, 256, 0, stream>>>(f, c, xs, dsh, child);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_column_table(const Levels& a, uint4* t, cudaStream_t stream) {
  const unsigned blocks = (unsigned)std::min<uint64_t>((std::max<uint64_t>(a.cap1, 1) + 255) / 256,
                                                       (uint64_t)device_sm_count() * 8);
  k_column_table<<<blocks, 256, 0, stream>>>(a, t);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_x_directory(const Levels& a, uint32_t* xdir, cudaStream_t stream) {
  const uint64_t n = (1ull << a.bits) + 1;
  const unsigned blocks = (unsigned)std::min<uint64_t>((n + 255) / 256,
                                                       (uint64_t)device_sm_count() * 8);
  k_x_directory<<<blocks, 256, 0, stream>>>(a, xdir);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_project_xy_device(const ProjPair* d_pairs, int S, uint64_t max_cap1,
                                  cudaStream_t stream) {
  if (S == 0) return cudaSuccess;
  const unsigned bx = (unsigned)std::min<uint64_t>((std::max<uint64_t>(max_cap1, 1) + 255) / 256, 64);
  k_project_xy_batch<<<dim3(bx, (unsigned)S), 256, 0, stream>>>(d_pairs);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace libcga
