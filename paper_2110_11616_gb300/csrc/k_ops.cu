// Operations on built CGAs: decode, merge, xy projection, exact NN search.
#include <algorithm>

#include "k_compact.cuh"

namespace libcga {

namespace {

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ decode
// Lossless inverse of the build: the walk X -> Y -> Z of Sec. III-A, done per
// tile of Z positions (each position finds its column and slab by binary
// search inside the tile's window).
__global__ void __launch_bounds__(kThreads) k_decode(Levels a, uint32_t* __restrict__ xyz) {
  __shared__ Window s_win;
  const uint32_t u = (uint32_t)a.hdr->cnt[0];
  const uint32_t start = blockIdx.x * kTile;
  if (start >= u) return;
  const uint32_t cnt = min((uint32_t)kTile, u - start);
  if (threadIdx.x == 0) {
    s_win = window_of(a, (uint32_t)a.hdr->cnt[1], (uint32_t)a.hdr->cnt[2], start, start + cnt - 1);
  }
  __syncthreads();
  const Window w = s_win;
  for (uint32_t e = threadIdx.x; e < cnt; e += kThreads) {
    uint32_t x, y, z;
    point_at(a, w, start + e, x, y, z);
    uint32_t* o = xyz + (size_t)(start + e) * 3;
    o[0] = x;
    o[1] = y;
    o[2] = z;
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

// Splitter keys: every half-th point of A, then of B.
__global__ void k_merge_spl(const MergePair* __restrict__ pairs, int S, uint32_t total,
                            uint32_t half, unsigned long long* spl) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const MergePair& P = pairs[find_pair_spl(pairs, S, i)];
  const uint32_t local = i - P.spl_base;
  const bool isA = local < P.spl_a;
  const Levels& L = isA ? P.a : P.b;
  const uint32_t k = isA ? local : local - P.spl_a;
  const uint32_t u = (uint32_t)L.hdr->cnt[0];
  const uint32_t pos = (k + 1) * half;
  spl[i] = (pos < u) ? key_at(L, (uint32_t)L.hdr->cnt[1], (uint32_t)L.hdr->cnt[2], pos)
                     : ~0ull;
}

// Tile bounds: each splitter s becomes the cut (rank_A(s), rank_B(s)) at its
// place in the key order of all splitters.
__global__ void k_merge_bounds(const MergePair* __restrict__ pairs, int S, uint32_t total,
                               uint32_t half, const unsigned long long* __restrict__ spl,
                               uint32_t* bounds) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int p = find_pair_spl(pairs, S, i);
  const MergePair& P = pairs[p];
  const uint32_t local = i - P.spl_base;
  const uint32_t uA = (uint32_t)P.a.hdr->cnt[0], uB = (uint32_t)P.b.hdr->cnt[0];
  const uint32_t NA = n_splitters(uA, P.spl_a, half), NB = n_splitters(uB, P.spl_b, half);
  const unsigned long long* sa = spl + P.spl_base;
  const unsigned long long* sb = sa + P.spl_a;
  const unsigned long long s = spl[i];
  uint32_t pos, ca, cb;
  if (local < P.spl_a) {
    const uint32_t k = local;
    if (k >= NA) return;
    uint32_t lo = 0, hi = NB;  // B splitters < s
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sb[mid] < s) lo = mid + 1; else hi = mid;
    }
    pos = k + lo;
    ca = (k + 1) * half;
    cb = rank_of(P.b, (uint32_t)P.b.hdr->cnt[2], s);
  } else {
    const uint32_t k = local - P.spl_a;
    if (k >= NB) return;
    uint32_t lo = 0, hi = NA;  // A splitters <= s
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sa[mid] <= s) lo = mid + 1; else hi = mid;
    }
    pos = k + lo;
    ca = rank_of(P.a, (uint32_t)P.a.hdr->cnt[2], s);
    cb = (k + 1) * half;
  }
  uint32_t* bnd = bounds + 2 * ((size_t)P.tile_base + p);
  bnd[2 * (pos + 1)] = ca;
  bnd[2 * (pos + 1) + 1] = cb;
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
  __shared__ CompactSmem sm;
  __shared__ Window s_wa, s_wb;
  __shared__ unsigned long long s_prev;
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
  if (tid == 0) {
    if (bad) atomicOr(&P.out.hdr->err, kErrInternal);
    if (na) s_wa = window_of(P.a, gA, hA, a0, a1 - 1);
    if (nb) s_wb = window_of(P.b, gB, hB, b0, b1 - 1);
    unsigned long long pk = 0;
    uint32_t has = 0;
    if (a0 > 0) {
      pk = key_at(P.a, gA, hA, a0 - 1);
      has = 1;
    }
    if (b0 > 0) {
      const unsigned long long kb = key_at(P.b, gB, hB, b0 - 1);
      pk = has ? max(pk, kb) : kb;
      has = 1;
    }
    s_prev = pk;
    s_has_prev = has;
  }
  __syncthreads();
  const uint32_t bA = P.a.bits;
  if (na) {
    const Window wa = s_wa;
    for (uint32_t e = tid; e < na; e += kThreads) {
      uint32_t x, y, z;
      point_at(P.a, wa, a0 + e, x, y, z);
      s_ab[e] = ((unsigned long long)x << (2 * bA)) | ((unsigned long long)y << bA) | z;
    }
  }
  if (nb) {
    const Window wb = s_wb;
    for (uint32_t e = tid; e < nb; e += kThreads) {
      uint32_t x, y, z;
      point_at(P.b, wb, b0 + e, x, y, z);
      s_ab[MH + e] = ((unsigned long long)x << (2 * bA)) | ((unsigned long long)y << bA) | z;
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

// ------------------------------------------------------------ x directory
// The dense per-x-value table of G-Arrays (Sec. III), here only as a lookup
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
  size_t b = 0;
  b += align_up((size_t)total_spl * 8);
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
  sc.spl = reinterpret_cast<unsigned long long*>(p);
  p += align_up((size_t)total_spl * 8);
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
  count_launch(total_spl > 0 ? 4 : 2);
  if (total_spl > 0) {
    k_merge_spl<<<(total_spl + 255) / 256, 256, 0, stream>>>(sc.pairs, S, total_spl, sc.half,
                                                            sc.spl);
    k_merge_bounds<<<(total_spl + 255) / 256, 256, 0, stream>>>(sc.pairs, S, total_spl, sc.half,
                                                               sc.spl, sc.bounds);
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
