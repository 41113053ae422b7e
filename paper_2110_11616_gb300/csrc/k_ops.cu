// Operations on built CGAs: decode, merge, xy projection, exact NN search.
#include <algorithm>
#include <atomic>

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
// Merge (Eq. 1, Sec. V-A) of pairs of CGAs in one grid, in tiles cut at
// column boundaries.  The (x, y) columns of both inputs are in key order (key
// x << b | y); a column present in both gets the union of its two sorted z
// lists, a column of one input keeps its z list.  Splitters sit at every
// `half`-th column of each input; a cut at column key s takes, from both
// inputs, the columns with key < s, so a column present in both never
// straddles two tiles and every tile can settle its columns alone.  A tile
// merges its voxels by (column key, z) keys (merge_tile_v), or, when its
// columns hold more voxels than shared memory stages, column by column
// (merge_tile); either way one packed block scan and one decoupled look-back
// over the pair's tiles give its voxel, column and slab offsets, and it
// writes its z entries, each output column's y and Y_pointer, and each new
// x's X_index and X_pointer entries.
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

// Splitters of an input with g columns (at most `reserved`).
__device__ __forceinline__ uint32_t n_splitters(uint32_t g, uint32_t reserved, uint32_t half) {
  const uint32_t k = g > 0 ? (g - 1) / half : 0u;
  return min(k, reserved);
}

// A tile bound: the first column of A and of B at or after the cut, and the
// slab holding each of them (h for the end of the input).
constexpr int kBoundWords = 4;

// Output header, empty-CGA sentinels, first and last tile bounds.
__global__ void k_merge_init(const MergePair* __restrict__ pairs, int S, uint32_t half,
                             uint32_t* bounds, uint32_t* ntiles) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S) return;
  const MergePair& P = pairs[p];
  const uint32_t gA = (uint32_t)P.a.hdr->cnt[1], gB = (uint32_t)P.b.hdr->cnt[1];
  const uint32_t hA = (uint32_t)P.a.hdr->cnt[2], hB = (uint32_t)P.b.hdr->cnt[2];
  const uint32_t NA = n_splitters(gA, P.spl_a, half), NB = n_splitters(gB, P.spl_b, half);
  const uint32_t nt = NA + NB + 1;
  ntiles[p] = nt;
  uint32_t* bnd = bounds + (size_t)kBoundWords * ((size_t)P.tile_base + p);
  bnd[0] = 0;
  bnd[1] = 0;
  bnd[2] = 0;
  bnd[3] = 0;
  bnd[kBoundWords * nt + 0] = gA;
  bnd[kBoundWords * nt + 1] = gB;
  bnd[kBoundWords * nt + 2] = hA;
  bnd[kBoundWords * nt + 3] = hB;
  P.out.hdr->cnt[0] = 0;
  P.out.hdr->cnt[1] = 0;
  P.out.hdr->cnt[2] = 0;
  P.out.hdr->err = P.a.hdr->err | P.b.hdr->err;
  P.out.ptr1[0] = 0;
  P.out.ptr2[0] = 0;
}

// Tile cuts, one warp per splitter.  Splitter k of A is A's column c = (k +
// 1) * half with key s; its cut is (c, #B columns < s), and its place among
// all splitters (A's before B's on equal keys) is k + #B splitters < s, where
// B splitter j (column (j + 1) * half) is below s exactly when (j + 1) * half
// < #B columns < s.  B's splitters mirror this, counting A's splitters with
// key <= s for the order but cutting A at key < s.  The ranks come from the
// Sec. V-A lookup at column level (x in X_index, then y in that slab).
__global__ void k_merge_cuts(const MergePair* __restrict__ pairs, int S, uint32_t total,
                             uint32_t half, uint32_t* bounds) {
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (i >= total) return;
  const int p = find_pair_spl(pairs, S, i);
  const MergePair& P = pairs[p];
  const uint32_t local = i - P.spl_base;
  const uint32_t gA = (uint32_t)P.a.hdr->cnt[1], gB = (uint32_t)P.b.hdr->cnt[1];
  const uint32_t NA = n_splitters(gA, P.spl_a, half), NB = n_splitters(gB, P.spl_b, half);
  const bool isA = local < P.spl_a;
  const uint32_t k = isA ? local : local - P.spl_a;
  if (k >= (isA ? NA : NB)) return;
  const Levels& own = isA ? P.a : P.b;
  const Levels& oth = isA ? P.b : P.a;
  const uint32_t hown = (uint32_t)own.hdr->cnt[2];
  const uint32_t goth = (uint32_t)oth.hdr->cnt[1], hoth = (uint32_t)oth.hdr->cnt[2];
  const uint32_t c = (k + 1) * half;  // < g of own
  const uint32_t s_own = warp_search_le(own.ptr2, 0, hown - 1, c);
  const uint32_t x = __ldg(own.idx2 + s_own), y = __ldg(own.idx1 + c);
  // #oth columns with key < (x, y), whether (x, y) is one, and the slab
  // holding the first column at or after the cut
  const uint32_t xr = warp_lower_bound_u16(oth.idx2, 0, hoth, x);
  uint32_t r = goth, slab_r = hoth;
  bool found = false;
  if (xr < hoth && __ldg(oth.idx2 + xr) == x) {
    const uint32_t ys = __ldg(oth.ptr2 + xr), ye = __ldg(oth.ptr2 + xr + 1);
    r = warp_lower_bound_u16(oth.idx1, ys, ye, y);
    found = r < ye && __ldg(oth.idx1 + r) == y;
    slab_r = r < ye ? xr : xr + 1;
  } else if (xr < hoth) {
    r = __ldg(oth.ptr2 + xr);
    slab_r = xr;
  }
  const uint32_t rk = isA ? r : r + (found ? 1u : 0u);
  const uint32_t before = rk > 0 ? min(isA ? NB : NA, (rk - 1) / half) : 0u;
  const uint32_t pos = k + before;
  if (lane == 0) {
    uint32_t* bnd = bounds + (size_t)kBoundWords * ((size_t)P.tile_base + p + pos + 1);
    bnd[0] = isA ? c : r;
    bnd[1] = isA ? r : c;
    bnd[2] = isA ? s_own : slab_r;
    bnd[3] = isA ? slab_r : s_own;
  }
}

// Size of the union of two ascending z lists (in shared or global memory).
__device__ __forceinline__ uint32_t union_count(const uint16_t* za, uint32_t na,
                                                const uint16_t* zb, uint32_t nb) {
  uint32_t i = 0, j = 0, n = 0;
  while (i < na && j < nb) {
    const uint32_t u = za[i], v = zb[j];
    i += u <= v;
    j += v <= u;
    ++n;
  }
  return n + (na - i) + (nb - j);
}

// Write the union of two ascending z lists to out.
__device__ __forceinline__ void union_write(const uint16_t* za, uint32_t na, const uint16_t* zb,
                                            uint32_t nb, uint16_t* __restrict__ out) {
  uint32_t i = 0, j = 0, n = 0;
  while (i < na && j < nb) {
    const uint32_t u = za[i], v = zb[j];
    out[n++] = (uint16_t)min(u, v);
    i += u <= v;
    j += v <= u;
  }
  while (i < na) out[n++] = za[i++];
  while (j < nb) out[n++] = zb[j++];
}

// z entries of each input the column-by-column tile path stages in shared
// memory (a tile whose columns hold more reads them from global memory).
template <int MH>
constexpr int merge_stage() { return MH == 2048 ? 1536 : 6144; }

// Voxels of each input the voxel-level tile path holds in shared memory (a
// tile with more on either side takes the column-by-column path).
template <int MH>
constexpr int merge_vstage() { return MH == 512 ? 1536 : (MH == 1024 ? 2560 : 2816); }

// Slabs of each input whose X_pointer and X_index entries the voxel-level
// tile path stages (a tile over more slabs searches them in global memory).
constexpr int kMergeSlabStage = 64;

// Shared memory of one merge tile: the larger of the two paths' layouts.
template <int MH>
constexpr size_t merge_col_bytes() { return 28 * (size_t)MH + 4 * (size_t)merge_stage<MH>() + 8; }
// voxel keys of both inputs, then one region holding first the staged
// Y_pointer, Y_index and slab entries and later the output z entries
template <int MH>
constexpr size_t merge_vox_stage_bytes() {
  return 8 * ((size_t)MH + 1) + 4 * (size_t)MH + 12 * (size_t)kMergeSlabStage;
}
template <int MH>
constexpr size_t merge_vox_bytes() {
  return 16 * (size_t)merge_vstage<MH>() +
         (4 * (size_t)merge_vstage<MH>() > merge_vox_stage_bytes<MH>() ? 4 * (size_t)merge_vstage<MH>()
                                                                        : merge_vox_stage_bytes<MH>());
}
template <int MH>
constexpr size_t merge_smem_bytes() {
  return ((merge_col_bytes<MH>() > merge_vox_bytes<MH>() ? merge_col_bytes<MH>()
                                                          : merge_vox_bytes<MH>()) + 15) & ~(size_t)15;
}

// Merge one tile of at most MH columns of each input (one splitter spacing)
// column by column: merge path over the column keys, then per output column
// its z list (a copy, or the union of two lists).  raw: merge_smem_bytes<MH>()
// bytes of shared memory, 16-byte aligned.
template <int MH>
__device__ __forceinline__ void merge_tile(const MergePair* __restrict__ pairs, int S,
                                           const uint32_t* __restrict__ bounds,
                                           const uint32_t* __restrict__ ntiles, uint32_t* clook,
                                           uint32_t t, int p, unsigned char* raw) {
  constexpr int IT = 2 * MH / kThreads;  // merged columns per thread
  static_assert(IT * kThreads == 2 * MH && MH % kThreads == 0, "merge tile shape");
  // merged keys; column keys of A and B; the tile's Y_pointer entries; merged
  // sources; staged z entries
  constexpr int ZS = merge_stage<MH>();
  uint32_t* s_mk = reinterpret_cast<uint32_t*>(raw);
  uint32_t* s_ka = s_mk + 2 * MH;
  uint32_t* s_kb = s_ka + MH;
  uint32_t* s_pa = s_kb + MH;
  uint32_t* s_pb = s_pa + MH + 1;
  uint16_t* s_ms = reinterpret_cast<uint16_t*>(s_pb + MH + 1);
  uint16_t* s_za = s_ms + 2 * MH;
  uint16_t* s_zb = s_za + ZS;
  __shared__ unsigned long long s_warp64[kWarps];
  __shared__ uint32_t s_tot[6], s_prevx, s_hasprev;
  const int tid = threadIdx.x;
  const MergePair& P = pairs[p];
  const uint32_t lt = t - P.tile_base;
  const uint32_t nt = ntiles[p];
  if (lt >= nt) return;
  const Levels &A = P.a, &B = P.b, &O = P.out;
  const uint32_t b = O.bits, ymask = (1u << b) - 1u;
  const uint32_t* bnd = bounds + (size_t)kBoundWords * ((size_t)P.tile_base + p + lt);
  const uint32_t a0 = bnd[0], b0 = bnd[1], sa0 = bnd[2], sb0 = bnd[3];
  const uint32_t a1 = bnd[4], b1 = bnd[5], sa1 = bnd[6], sb1 = bnd[7];
  uint32_t na = a1 - a0, nb = b1 - b0;
  const bool bad = a1 < a0 || b1 < b0 || na > (uint32_t)MH || nb > (uint32_t)MH;
  if (bad) {
    na = 0;
    nb = 0;
  }
  // the slab of the tile's last column: the slab of the next tile's first
  // column, one less when that column opens its slab
  const uint32_t saL = na ? (__ldg(A.ptr2 + sa1) == a1 ? sa1 - 1 : sa1) : sa0;
  const uint32_t sbL = nb ? (__ldg(B.ptr2 + sb1) == b1 ? sb1 - 1 : sb1) : sb0;
  if (tid == 0) {
    if (bad) atomicOr(&O.hdr->err, kErrInternal);
    // x of the column just before the tile (the larger of A's and B's)
    uint32_t px = 0, pk = 0;
    const bool hp = a0 > 0 || b0 > 0;
    if (a0 > 0) {
      const uint32_t s = __ldg(A.ptr2 + sa0) == a0 ? sa0 - 1 : sa0;
      pk = ((uint32_t)__ldg(A.idx2 + s) << b) | __ldg(A.idx1 + a0 - 1);
    }
    if (b0 > 0) {
      const uint32_t s = __ldg(B.ptr2 + sb0) == b0 ? sb0 - 1 : sb0;
      pk = max(pk, ((uint32_t)__ldg(B.idx2 + s) << b) | __ldg(B.idx1 + b0 - 1));
    }
    px = pk >> b;
    s_prevx = px;
    s_hasprev = hp ? 1u : 0u;
  }
  // column keys: each column's slab by a search of the tile's few slabs
  // (their X_pointer entries stay in L1)
  for (uint32_t e = tid; e < na; e += kThreads) {
    const uint32_t sl = search_le(A.ptr2, sa0, saL, a0 + e);
    s_ka[e] = ((uint32_t)__ldg(A.idx2 + sl) << b) | __ldg(A.idx1 + a0 + e);
  }
  for (uint32_t e = tid; e < nb; e += kThreads) {
    const uint32_t sl = search_le(B.ptr2, sb0, sbL, b0 + e);
    s_kb[e] = ((uint32_t)__ldg(B.idx2 + sl) << b) | __ldg(B.idx1 + b0 + e);
  }
  // the tile's z entries of each input are one contiguous range: staged in
  // shared memory by coalesced loads when they fit
  const uint32_t zA0 = na ? __ldg(A.ptr1 + a0) : 0u, zA1 = na ? __ldg(A.ptr1 + a1) : 0u;
  const uint32_t zB0 = nb ? __ldg(B.ptr1 + b0) : 0u, zB1 = nb ? __ldg(B.ptr1 + b1) : 0u;
  const bool stA = zA1 - zA0 <= (uint32_t)ZS, stB = zB1 - zB0 <= (uint32_t)ZS;
  if (stA) {
    for (uint32_t e = tid; e < zA1 - zA0; e += kThreads) s_za[e] = __ldg(A.idx0 + zA0 + e);
  }
  if (stB) {
    for (uint32_t e = tid; e < zB1 - zB0; e += kThreads) s_zb[e] = __ldg(B.idx0 + zB0 + e);
  }
  const uint16_t* zAb = stA ? s_za - zA0 : A.idx0;  // z entry i of A at zAb[i]
  const uint16_t* zBb = stB ? s_zb - zB0 : B.idx0;
  // Y_pointer of the tile's columns (and the one after), column i of A at
  // pA[i] (i relative to a0)
  for (uint32_t e = tid; e <= na; e += kThreads) s_pa[e] = na ? __ldg(A.ptr1 + a0 + e) : 0u;
  for (uint32_t e = tid; e <= nb; e += kThreads) s_pb[e] = nb ? __ldg(B.ptr1 + b0 + e) : 0u;
  __syncthreads();
  // merge path (A first on equal keys); sources: A's column i as i, B's
  // column j as MH + j
  const uint32_t n = na + nb;
  const uint32_t diag = min((uint32_t)(tid * IT), n);
  {
    uint32_t lo = diag > nb ? diag - nb : 0u, hi = min(diag, na);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_ka[mid] <= s_kb[diag - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    uint32_t i = lo, j = diag - lo;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      if (diag + it >= n) break;
      const bool takeA = i < na && (j >= nb || s_ka[i] <= s_kb[j]);
      s_mk[diag + it] = takeA ? s_ka[i] : s_kb[j];
      s_ms[diag + it] = (uint16_t)(takeA ? i : MH + j);
      if (takeA) ++i; else ++j;
    }
  }
  __syncthreads();
  // output columns: a merged key that differs from the one before it; a key
  // present in both inputs appears twice in a row (A's, then B's)
  const uint32_t prevx = s_prevx;
  const bool hasprev = s_hasprev != 0;
  uint32_t cnt[IT];
  uint32_t nv = 0, nh = 0, ns = 0;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    cnt[it] = 0;
    const uint32_t ps = diag + it;
    if (ps >= n) continue;
    const uint32_t key = s_mk[ps];
    if (ps > 0 && s_mk[ps - 1] == key) continue;  // B's copy of a shared column
    const uint32_t src = s_ms[ps];
    const bool pair = ps + 1 < n && s_mk[ps + 1] == key;
    uint32_t c;
    if (pair) {
      const uint32_t ia = src, ib = s_ms[ps + 1] - MH;
      const uint32_t za = s_pa[ia], zb = s_pb[ib];
      c = union_count(zAb + za, s_pa[ia + 1] - za, zBb + zb, s_pb[ib + 1] - zb);
    } else if (src < MH) {
      c = s_pa[src + 1] - s_pa[src];
    } else {
      c = s_pb[src - MH + 1] - s_pb[src - MH];
    }
    cnt[it] = c;
    const uint32_t x = key >> b;
    const bool newslab = ps > 0 ? (s_mk[ps - 1] >> b) != x : (!hasprev || x != prevx);
    nv += c;
    ++nh;
    ns += newslab ? 1u : 0u;
  }
  // one block scan of (voxels | columns << 32 | slabs << 48): a tile holds at
  // most 2 * MH <= 4096 columns and slabs and fewer than 2^32 voxels
  unsigned long long tp = 0;
  const unsigned long long op = block_excl_scan<unsigned long long>(
      (unsigned long long)nv | ((unsigned long long)nh << 32) | ((unsigned long long)ns << 48),
      tp, s_warp64);
  const uint32_t ov = (uint32_t)op, ohs = (uint32_t)(op >> 32);
  const uint32_t tv = (uint32_t)tp, thc = (uint32_t)(tp >> 32);
  if (tid < 3) {
    const uint32_t run = tid == 0 ? tv : (tid == 1 ? (thc & 0xffffu) : (thc >> 16));
    uint32_t* my = clook + (size_t)t * 3 + tid;
    uint32_t excl = 0;
    if (lt == 0) {
      st_relaxed(my, kFlagInc | run);
    } else {
      st_relaxed(my, kFlagAgg | run);
      excl = lookback(clook + tid, 3, t, P.tile_base, &O.hdr->err);
      st_relaxed(my, kFlagInc | ((excl + run) & kValMask));
    }
    s_tot[tid] = excl;
    s_tot[3 + tid] = excl + run;
  }
  __syncthreads();
  uint32_t vo = s_tot[0] + ov, co = s_tot[1] + (ohs & 0xffffu), so = s_tot[2] + (ohs >> 16);
  bool over = false;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const uint32_t ps = diag + it;
    if (ps >= n) continue;
    const uint32_t key = s_mk[ps];
    if (ps > 0 && s_mk[ps - 1] == key) continue;
    const uint32_t src = s_ms[ps];
    const bool pair = ps + 1 < n && s_mk[ps + 1] == key;
    const uint32_t c = cnt[it];
    if (co >= O.cap1 || vo + c > O.cap) {
      over = true;
      continue;
    }
    O.idx1[co] = (uint16_t)(key & ymask);
    O.ptr1[co] = vo;
    if (pair) {
      const uint32_t ia = src, ib = s_ms[ps + 1] - MH;
      const uint32_t za = s_pa[ia], zb = s_pb[ib];
      union_write(zAb + za, s_pa[ia + 1] - za, zBb + zb, s_pb[ib + 1] - zb, O.idx0 + vo);
    } else {
      const bool fromA = src < MH;
      const uint16_t* zz = fromA ? zAb + s_pa[src] : zBb + s_pb[src - MH];
      for (uint32_t q = 0; q < c; ++q) O.idx0[vo + q] = zz[q];
    }
    const uint32_t x = key >> b;
    const bool newslab = ps > 0 ? (s_mk[ps - 1] >> b) != x : (!hasprev || x != prevx);
    if (newslab) {
      if (so < O.cap2) {
        O.idx2[so] = (uint16_t)x;
        O.ptr2[so] = co;
      } else {
        over = true;
      }
      ++so;
    }
    vo += c;
    ++co;
  }
  if (over) atomicOr(&O.hdr->err, kErrInternal);
  if (lt == nt - 1 && tid == 0) {
    const uint32_t U = s_tot[3], G = s_tot[4], H = s_tot[5];
    if (G <= O.cap1) O.ptr1[G] = U;
    if (H <= O.cap2) O.ptr2[H] = G;
    O.hdr->cnt[0] = U;
    O.hdr->cnt[1] = G;
    O.hdr->cnt[2] = H;
  }
}

// Next tile id for a resident block (total_tiles when none is left).  A
// reserved tile at or beyond its pair's actual count means the pair's later
// ones hold nothing either: the counter jumps to the next pair's first tile,
// and after the last pair the block stops.  Each round moves to a later pair,
// and real tiles still go out in increasing order.
__device__ __forceinline__ uint32_t next_merge_tile(const MergePair* __restrict__ pairs, int S,
                                                    const uint32_t* __restrict__ ntiles,
                                                    uint32_t* counter, uint32_t total_tiles,
                                                    int& p) {
  for (;;) {
    const uint32_t t = atomicAdd(counter, 1u);
    p = 0;
    if (t >= total_tiles) return total_tiles;
    p = find_pair_tile(pairs, S, t);
    if (t - pairs[p].tile_base < ntiles[p]) return t;
    if (p + 1 >= S) {
      p = 0;
      return total_tiles;
    }
    atomicMax(counter, pairs[p + 1].tile_base);
  }
}

// Merge one tile voxel by voxel.  Each voxel of the tile gets its full key
// (x << b | y) << 16 | z; both key runs are ascending, so the tile's output is
// their merge with equal keys (a voxel present in both inputs, adjacent in the
// merge) kept once.  Merge path splits the tile's voxels evenly over the
// threads whatever the columns hold; an output voxel opens a column when its
// column key differs from the previous output voxel's, and a slab when its x
// does.  One block scan of (voxels, columns, slabs) and the look-back give the
// tile's offsets; z entries go out through shared memory in one coalesced
// pass, column and slab entries straight from the walk.  A tile with more than
// merge_vstage<MH>() voxels on either side (dense columns) takes the
// column-by-column path instead.
template <int MH>
__device__ __forceinline__ void merge_tile_v(const MergePair* __restrict__ pairs, int S,
                                             const uint32_t* __restrict__ bounds,
                                             const uint32_t* __restrict__ ntiles, uint32_t* clook,
                                             uint32_t t, int p, unsigned char* raw) {
  constexpr int VS = merge_vstage<MH>();
  static_assert(2 * VS <= 32 * kThreads, "a thread's merged voxels fit one 32-bit mask");
  constexpr unsigned long long kF = (1ull << 21) - 1ull;  // one field of the packed scan
  __shared__ unsigned long long s_w64[kWarps];
  __shared__ uint32_t s_vt[6], s_vprevck, s_vhasprev;
  const int tid = threadIdx.x;
  const MergePair& P = pairs[p];
  const uint32_t lt = t - P.tile_base;
  const uint32_t nt = ntiles[p];
  if (lt >= nt) return;
  const Levels &A = P.a, &B = P.b, &O = P.out;
  const uint32_t b = O.bits, ymask = (1u << b) - 1u;
  const uint32_t* bnd = bounds + (size_t)kBoundWords * ((size_t)P.tile_base + p + lt);
  const uint32_t a0 = bnd[0], b0 = bnd[1], sa0 = bnd[2], sb0 = bnd[3];
  const uint32_t a1 = bnd[4], b1 = bnd[5], sa1 = bnd[6], sb1 = bnd[7];
  const uint32_t na = a1 - a0, nb = b1 - b0;
  const bool bad = a1 < a0 || b1 < b0 || na > (uint32_t)MH || nb > (uint32_t)MH;
  uint32_t zA0 = 0, zA1 = 0, zB0 = 0, zB1 = 0;
  if (!bad) {
    if (na) {
      zA0 = __ldg(A.ptr1 + a0);
      zA1 = __ldg(A.ptr1 + a1);
    }
    if (nb) {
      zB0 = __ldg(B.ptr1 + b0);
      zB1 = __ldg(B.ptr1 + b1);
    }
  }
  const uint32_t nva = zA1 - zA0, nvb = zB1 - zB0;  // wraps (and so falls back) if corrupt
  if (bad || nva > (uint32_t)VS || nvb > (uint32_t)VS) {
    merge_tile<MH>(pairs, S, bounds, ntiles, clook, t, p, raw);
    return;
  }
  unsigned long long* s_va = reinterpret_cast<unsigned long long*>(raw);
  unsigned long long* s_vb = s_va + VS;
  uint16_t* s_oz = reinterpret_cast<uint16_t*>(s_vb + VS);  // 2 * VS output z entries
  // staged entries of the tile's columns and slabs (the same region as s_oz)
  uint32_t* s_pa = reinterpret_cast<uint32_t*>(s_vb + VS);  // Y_pointer, na + 1
  uint32_t* s_pb = s_pa + MH + 1;
  uint16_t* s_ya = reinterpret_cast<uint16_t*>(s_pb + MH + 1);  // Y_index, na
  uint16_t* s_yb = s_ya + MH;
  uint32_t* s_xpa = reinterpret_cast<uint32_t*>(s_yb + MH);  // X_pointer of the slabs
  uint32_t* s_xpb = s_xpa + kMergeSlabStage;
  uint16_t* s_xa = reinterpret_cast<uint16_t*>(s_xpb + kMergeSlabStage);  // X_index
  uint16_t* s_xb = s_xa + kMergeSlabStage;
  const uint32_t saL = na ? (__ldg(A.ptr2 + sa1) == a1 ? sa1 - 1 : sa1) : sa0;
  const uint32_t sbL = nb ? (__ldg(B.ptr2 + sb1) == b1 ? sb1 - 1 : sb1) : sb0;
  const uint32_t nsa = na ? saL - sa0 + 1 : 0u, nsb = nb ? sbL - sb0 + 1 : 0u;
  const bool xsa = nsa <= (uint32_t)kMergeSlabStage, xsb = nsb <= (uint32_t)kMergeSlabStage;
  if (tid == 0) {
    // key of the column just before the tile (the larger of A's and B's)
    uint32_t pk = 0;
    if (a0 > 0) {
      const uint32_t s = __ldg(A.ptr2 + sa0) == a0 ? sa0 - 1 : sa0;
      pk = ((uint32_t)__ldg(A.idx2 + s) << b) | __ldg(A.idx1 + a0 - 1);
    }
    if (b0 > 0) {
      const uint32_t s = __ldg(B.ptr2 + sb0) == b0 ? sb0 - 1 : sb0;
      pk = max(pk, ((uint32_t)__ldg(B.idx2 + s) << b) | __ldg(B.idx1 + b0 - 1));
    }
    s_vprevck = pk;
    s_vhasprev = (a0 > 0 || b0 > 0) ? 1u : 0u;
  }
  // stage the tile's z entries (the low bits of the voxel keys), Y_pointer
  // and Y_index entries and its slabs' entries: independent coalesced loads
  for (uint32_t e = tid; e < nva; e += kThreads) s_va[e] = __ldg(A.idx0 + zA0 + e);
  for (uint32_t e = tid; e < nvb; e += kThreads) s_vb[e] = __ldg(B.idx0 + zB0 + e);
  if (na) {
    for (uint32_t e = tid; e <= na; e += kThreads) s_pa[e] = __ldg(A.ptr1 + a0 + e);
    for (uint32_t e = tid; e < na; e += kThreads) s_ya[e] = __ldg(A.idx1 + a0 + e);
  }
  if (nb) {
    for (uint32_t e = tid; e <= nb; e += kThreads) s_pb[e] = __ldg(B.ptr1 + b0 + e);
    for (uint32_t e = tid; e < nb; e += kThreads) s_yb[e] = __ldg(B.idx1 + b0 + e);
  }
  if (xsa) {
    for (uint32_t e = tid; e < nsa; e += kThreads) {
      s_xpa[e] = __ldg(A.ptr2 + sa0 + e);
      s_xa[e] = __ldg(A.idx2 + sa0 + e);
    }
  }
  if (xsb) {
    for (uint32_t e = tid; e < nsb; e += kThreads) {
      s_xpb[e] = __ldg(B.ptr2 + sb0 + e);
      s_xb[e] = __ldg(B.idx2 + sb0 + e);
    }
  }
  __syncthreads();
  // voxel keys: each column's key (its slab by a search of the tile's slabs)
  // over its Y_pointer range, clamped to the tile's z range
  for (uint32_t e = tid; e < na; e += kThreads) {
    uint32_t x;
    if (xsa) {
      uint32_t lo = 0, hi = nsa - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (s_xpa[mid] <= a0 + e) lo = mid; else hi = mid - 1;
      }
      x = s_xa[lo];
    } else {
      x = __ldg(A.idx2 + search_le(A.ptr2, sa0, saL, a0 + e));
    }
    const unsigned long long ck = (unsigned long long)((x << b) | s_ya[e]) << 16;
    const uint32_t q0 = max(s_pa[e], zA0), q1 = min(s_pa[e + 1], zA1);
    for (uint32_t q = q0; q < q1; ++q) s_va[q - zA0] |= ck;
  }
  for (uint32_t e = tid; e < nb; e += kThreads) {
    uint32_t x;
    if (xsb) {
      uint32_t lo = 0, hi = nsb - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (s_xpb[mid] <= b0 + e) lo = mid; else hi = mid - 1;
      }
      x = s_xb[lo];
    } else {
      x = __ldg(B.idx2 + search_le(B.ptr2, sb0, sbL, b0 + e));
    }
    const unsigned long long ck = (unsigned long long)((x << b) | s_yb[e]) << 16;
    const uint32_t q0 = max(s_pb[e], zB0), q1 = min(s_pb[e + 1], zB1);
    for (uint32_t q = q0; q < q1; ++q) s_vb[q - zB0] |= ck;
  }
  __syncthreads();
  // merge path over the tile's voxels (A first on equal keys), the same
  // number of merged positions for every thread
  const uint32_t nv = nva + nvb;
  const uint32_t per = (nv + kThreads - 1) / kThreads;
  const uint32_t diag = min(tid * per, nv), dend = min(diag + per, nv);
  uint32_t i0, j0;
  {
    uint32_t lo = diag > nvb ? diag - nvb : 0u, hi = min(diag, nva);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_va[mid] <= s_vb[diag - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    i0 = lo;
    j0 = diag - lo;
  }
  // the merged voxel before the thread's first one: the larger of the last
  // taken of A and of B; before the tile's first voxel, a key whose column
  // differs and whose x differs exactly when no column precedes the tile or
  // the preceding column's x differs
  unsigned long long pk0;
  if (diag > 0) {
    pk0 = 0;
    if (i0 > 0) pk0 = s_va[i0 - 1];
    if (j0 > 0) pk0 = max(pk0, s_vb[j0 - 1]);
  } else {
    pk0 = s_vhasprev ? (((unsigned long long)s_vprevck << 16) | 0xffffull) : ~0ull;
  }
  // first walk: the merge decisions and, against the previous merged key,
  // whether each voxel is new (not B's copy of A's), opens a column, opens a
  // slab; kept as bit masks for the second walk
  const uint32_t cnt = dend - diag;  // at most 32
  const uint32_t sh = 16 + b;
  uint32_t mA = 0, mU = 0, mC = 0, mS = 0, cv = 0, cc = 0, cs = 0;
  {
    uint32_t i = i0, j = j0;
    unsigned long long ka = i < nva ? s_va[i] : ~0ull, kb = j < nvb ? s_vb[j] : ~0ull, pk = pk0;
    for (uint32_t q = 0; q < cnt; ++q) {
      const bool takeA = ka <= kb;  // keys are below 2^48: ~0 marks an input used up
      const unsigned long long k = takeA ? ka : kb;
      if (takeA) {
        ++i;
        ka = i < nva ? s_va[i] : ~0ull;
      } else {
        ++j;
        kb = j < nvb ? s_vb[j] : ~0ull;
      }
      const unsigned long long d = k ^ pk;
      const uint32_t u = d != 0ull, c = (d >> 16) != 0ull, sl = (d >> sh) != 0ull;
      mA |= (uint32_t)takeA << q;
      mU |= u << q;
      mC |= c << q;
      mS |= sl << q;
      cv += u;
      cc += c;
      cs += sl;
      pk = k;
    }
  }
  unsigned long long tp = 0;
  const unsigned long long op = block_excl_scan<unsigned long long>(
      (unsigned long long)cv | ((unsigned long long)cc << 21) | ((unsigned long long)cs << 42), tp,
      s_w64);
  if (tid < 3) {
    const uint32_t run = (uint32_t)((tp >> (21 * tid)) & kF);
    uint32_t* my = clook + (size_t)t * 3 + tid;
    uint32_t excl = 0;
    if (lt == 0) {
      st_relaxed(my, kFlagInc | run);
    } else {
      st_relaxed(my, kFlagAgg | run);
      excl = lookback(clook + tid, 3, t, P.tile_base, &O.hdr->err);
      st_relaxed(my, kFlagInc | ((excl + run) & kValMask));
    }
    s_vt[tid] = excl;
    s_vt[3 + tid] = excl + run;
  }
  __syncthreads();
  // second walk, replaying the masks: z entries to shared memory, column and
  // slab entries out
  const uint32_t vo0 = s_vt[0], co0 = s_vt[1], so0 = s_vt[2];
  bool over = false;
  {
    uint32_t o = (uint32_t)(op & kF), c = co0 + (uint32_t)((op >> 21) & kF),
             sx = so0 + (uint32_t)(op >> 42);
    uint32_t i = i0, j = j0;
    for (uint32_t q = 0; q < cnt; ++q) {
      const bool takeA = (mA >> q) & 1u;
      const unsigned long long k = *(takeA ? s_va + i : s_vb + j);
      i += takeA ? 1u : 0u;
      j += takeA ? 0u : 1u;
      if (!((mU >> q) & 1u)) continue;
      s_oz[o] = (uint16_t)k;
      if ((mC >> q) & 1u) {
        const uint32_t col = (uint32_t)(k >> 16);
        if ((mS >> q) & 1u) {
          if (sx < O.cap2) {
            O.idx2[sx] = (uint16_t)(col >> b);
            O.ptr2[sx] = c;
          } else {
            over = true;
          }
          ++sx;
        }
        if (c < O.cap1) {
          O.idx1[c] = (uint16_t)(col & ymask);
          O.ptr1[c] = vo0 + o;
        } else {
          over = true;
        }
        ++c;
      }
      ++o;
    }
  }
  __syncthreads();
  const uint32_t nu = (uint32_t)(tp & kF);
  for (uint32_t e = tid; e < nu; e += kThreads) {
    if (vo0 + e < O.cap) O.idx0[vo0 + e] = s_oz[e]; else over = true;
  }
  if (over) atomicOr(&O.hdr->err, kErrInternal);
  if (lt == nt - 1 && tid == 0) {
    const uint32_t U = s_vt[3], G = s_vt[4], H = s_vt[5];
    if (G <= O.cap1) O.ptr1[G] = U;
    if (H <= O.cap2) O.ptr2[H] = G;
    O.hdr->cnt[0] = U;
    O.hdr->cnt[1] = G;
    O.hdr->cnt[2] = H;
  }
}

// Merge tiles by the resident blocks: each takes tile ids from the counter in
// launch order until the reserved tiles are handed out (tiles beyond a
// pair's actual count are skipped), so the look-back always finds its
// predecessors running or done.
template <int MH>
__global__ void __launch_bounds__(kThreads, 4) k_merge_tiles(const MergePair* __restrict__ pairs,
                                                          int S, const uint32_t* __restrict__ bounds,
                                                          const uint32_t* __restrict__ ntiles,
                                                          uint32_t* clook, uint32_t* counter,
                                                          uint32_t total_tiles) {
  __shared__ __align__(16) unsigned char s_raw[merge_smem_bytes<MH>()];
  __shared__ uint32_t s_tile;
  __shared__ int s_p;
  for (;;) {
    __syncthreads();  // the previous tile's shared data is read no more
    if (threadIdx.x == 0) {
      int p;
      s_tile = next_merge_tile(pairs, S, ntiles, counter, total_tiles, p);
      s_p = p;
    }
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= total_tiles) return;
    merge_tile_v<MH>(pairs, S, bounds, ntiles, clook, t, s_p, s_raw);
  }
}

// ---------------------------------------------------------- key-level merge
// On fine grids (14 or more bits per axis) a column holds about one voxel, so
// the column-level merge has nothing to gain; there the two sorted key
// sequences are merged directly: splitters at every half-th point of each
// input, each tile decodes both runs into 64-bit keys in shared memory
// (window expansion), merges them by merge path and re-compacts them.
__device__ __forceinline__ uint32_t n_splitters_pts(uint32_t u, uint32_t reserved, uint32_t half) {
  const uint32_t k = u > 0 ? (u - 1) / half : 0u;
  return min(k, reserved);
}

// Key-level merge (fine grids): output header, empty-CGA sentinels, first and
// last tile bounds (two words per bound: the first point of A and of B).
__global__ void k_kmerge_init(const MergePair* __restrict__ pairs, int S, uint32_t half,
                             uint32_t* bounds, uint32_t* ntiles) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S) return;
  const MergePair& P = pairs[p];
  const uint32_t uA = (uint32_t)P.a.hdr->cnt[0], uB = (uint32_t)P.b.hdr->cnt[0];
  const uint32_t NA = n_splitters_pts(uA, P.spl_a, half), NB = n_splitters_pts(uB, P.spl_b, half);
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

// Key-level merge: tile cuts, one warp per splitter.  Splitter k of A is A's key s at
// position (k + 1) * half; its cut is (rank_A(s), rank_B(s)) = ((k + 1) *
// half, #B keys < s), and its place among all splitters (A's before B's on
// equal keys) is k + #B splitters < s, where B splitter j (the key at
// (j + 1) * half) is below s exactly when (j + 1) * half < rank_B(s).  B's
// splitters mirror this with #A keys <= s.  The Sec. V-A lookup gives the
// ranks.
__global__ void k_kmerge_cuts(const MergePair* __restrict__ pairs, int S, uint32_t total,
                             uint32_t half, uint32_t* bounds) {
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (i >= total) return;
  const int p = find_pair_spl(pairs, S, i);
  const MergePair& P = pairs[p];
  const uint32_t local = i - P.spl_base;
  const uint32_t uA = (uint32_t)P.a.hdr->cnt[0], uB = (uint32_t)P.b.hdr->cnt[0];
  const uint32_t NA = n_splitters_pts(uA, P.spl_a, half), NB = n_splitters_pts(uB, P.spl_b, half);
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

// Key-level merge of one tile: decode both runs (at most MH points each) into shared
// memory, merge-path split per thread, sequential merge, then the shared
// dedupe + compaction.
template <int MH>
__device__ __forceinline__ void kmerge_tile(const MergePair* __restrict__ pairs, int S,
                                            const uint32_t* __restrict__ bounds,
                                            const uint32_t* __restrict__ ntiles, uint32_t* clook,
                                            uint32_t t, int p) {
  constexpr int IT = 2 * MH / kThreads;  // merged keys per thread
  static_assert(IT * kThreads == 2 * MH && 2 * MH <= kTile, "merge tile shape");
  __shared__ unsigned long long s_ab[2 * MH];
  __shared__ uint16_t s_col[MH], s_slab[MH];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ CompactSmem sm;
  __shared__ Window s_wa, s_wb;
  __shared__ unsigned long long s_prev, s_prev2[2];
  __shared__ uint32_t s_has_prev;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
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

// Key-level merge tiles by the resident blocks (as k_merge_tiles).
template <int MH>
__global__ void __launch_bounds__(kThreads, 4) k_kmerge_tiles(const MergePair* __restrict__ pairs,
                                                           int S, const uint32_t* __restrict__ bounds,
                                                           const uint32_t* __restrict__ ntiles,
                                                           uint32_t* clook, uint32_t* counter,
                                                           uint32_t total_tiles) {
  __shared__ uint32_t s_tile;
  __shared__ int s_p;
  for (;;) {
    __syncthreads();  // the previous tile's shared data is read no more
    if (threadIdx.x == 0) {
      int p;
      s_tile = next_merge_tile(pairs, S, ntiles, counter, total_tiles, p);
      s_p = p;
    }
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= total_tiles) return;
    kmerge_tile<MH>(pairs, S, bounds, ntiles, clook, t, s_p);
  }
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

// ------------------------------------------------------ bitmap projection
// The xz or yz projection (Eq. 3) of a CGA on a grid of 5 to 13 bits per axis
// without a sort: one bit per 2D voxel (2^(2b) bits, row = the kept first
// axis, column = z) is set for every stored voxel, and the set bits read row
// by row, in order, are the distinct 2D voxels in key order: U_index the
// non-empty rows, V_index the set columns of each.

// Set the bits of a's voxels (a tile of Z positions per block, decoded by the
// X -> Y -> Z walk of Sec. V-A as in k_decode).
__global__ void __launch_bounds__(kThreads) k_proj_set(Levels a, int plane,
                                                       uint32_t* __restrict__ bits) {
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
  const uint32_t b = a.bits;
  for (uint32_t e = threadIdx.x; e < cnt; e += kThreads) {
    const uint32_t cr = s_col[e];
    const uint32_t r = plane == 1 ? (uint32_t)__ldg(a.idx2 + w.x0 + s_slab[cr])
                                  : (uint32_t)__ldg(a.idx1 + w.c0 + cr);
    const uint32_t key = (r << b) | __ldg(a.idx0 + start + e);
    atomicOr(bits + (key >> 5), 1u << (key & 31u));
  }
}

// Set bits of each row: one warp per row, each lane a run of the row's words.
__global__ void __launch_bounds__(256) k_proj_rows(const uint32_t* __restrict__ bits, uint32_t b,
                                                   uint32_t* __restrict__ rowcnt) {
  const uint32_t row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
  if (row >= (1u << b)) return;
  const uint32_t words = 1u << (b - 5), per = words > 32u ? words / 32u : 1u;
  const uint32_t* rw = bits + (size_t)row * words;
  uint32_t c = 0;
  for (uint32_t k = 0; k < per; ++k) {
    const uint32_t wi = lane * per + k;
    if (wi < words) c += (uint32_t)__popc(__ldg(rw + wi));
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) rowcnt[row] = c;
}

// Row offsets (exclusive scan of the row counts) and the U arrays, by one
// block: thread i takes rows [i * per, (i + 1) * per).
__global__ void __launch_bounds__(kThreads) k_proj_scan(const uint32_t* __restrict__ rowcnt,
                                                        uint32_t b, uint32_t* __restrict__ rowoff,
                                                        Levels o, const Header* __restrict__ src) {
  __shared__ unsigned long long s_warp[kWarps];
  const uint32_t rows = 1u << b, per = (rows + kThreads - 1) / kThreads;
  const uint32_t r0 = threadIdx.x * per;
  uint32_t v = 0, ne = 0;
  for (uint32_t k = 0; k < per && r0 + k < rows; ++k) {
    const uint32_t c = rowcnt[r0 + k];
    v += c;
    ne += c != 0u;
  }
  // voxels in the low word, non-empty rows in the high word
  unsigned long long tot = 0;
  const unsigned long long ex = block_excl_scan<unsigned long long>(
      (unsigned long long)v | ((unsigned long long)ne << 32), tot, s_warp);
  uint32_t off = (uint32_t)ex, ui = (uint32_t)(ex >> 32);
  for (uint32_t k = 0; k < per && r0 + k < rows; ++k) {
    const uint32_t r = r0 + k, c = rowcnt[r];
    rowoff[r] = off;
    if (c != 0u) {
      o.idx1[ui] = (uint16_t)r;
      o.ptr1[ui] = off;
      ++ui;
    }
    off += c;
  }
  if (threadIdx.x == 0) {
    const uint32_t total = (uint32_t)tot, h = (uint32_t)(tot >> 32);
    o.ptr1[h] = total;
    o.hdr->cnt[0] = total;
    o.hdr->cnt[1] = h;
    o.hdr->cnt[2] = 0;
    o.hdr->err = src->err;
  }
}

// V_index: the set columns of each row in order (one warp per row).
__global__ void __launch_bounds__(256) k_proj_write(const uint32_t* __restrict__ bits, uint32_t b,
                                                    const uint32_t* __restrict__ rowoff, Levels o) {
  const uint32_t row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
  if (row >= (1u << b)) return;
  const uint32_t words = 1u << (b - 5), per = words > 32u ? words / 32u : 1u;
  const uint32_t* rw = bits + (size_t)row * words;
  uint32_t c = 0;
  for (uint32_t k = 0; k < per; ++k) {
    const uint32_t wi = lane * per + k;
    if (wi < words) c += (uint32_t)__popc(__ldg(rw + wi));
  }
  // the lane's first output position: the row's offset and the set bits of
  // the lanes before it
  uint32_t incl = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += x;
  }
  uint32_t pos = __ldg(rowoff + row) + incl - c;
  for (uint32_t k = 0; k < per; ++k) {
    const uint32_t wi = lane * per + k;
    if (wi >= words) break;
    for (uint32_t m = __ldg(rw + wi); m != 0u; m &= m - 1u) {
      o.idx0[pos++] = (uint16_t)(wi * 32u + (uint32_t)__ffs((int)m) - 1u);
    }
  }
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
  b += align_up(((size_t)total_tiles + S) * kBoundWords * 4 + 16);
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
  p += align_up(((size_t)total_tiles + S) * kBoundWords * 4 + 16);
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

// Resident blocks of a merge tile kernel on the device (queried once per
// kernel), the grid of its persistent launch.
template <typename F>
static uint32_t merge_grid(F* kernel, std::atomic<int>& cache, uint32_t total_tiles) {
  int n = cache.load(std::memory_order_relaxed);
  if (n == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, 0) != cudaSuccess ||
        n <= 0) {
      cudaGetLastError();
      n = 2;
    }
    cache.store(n, std::memory_order_relaxed);
  }
  return std::max<uint32_t>(1u, std::min<uint32_t>(total_tiles, (uint32_t)(n * device_sm_count())));
}

cudaError_t run_merge_device(int S, uint32_t total_spl, uint32_t total_tiles,
                             const MergeScratch& sc, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(sc.clook, 0, sc.zero_bytes, stream);
  if (e != cudaSuccess) return e;
  if (sc.half != 512 && sc.half != 1024 && sc.half != 2048) return cudaErrorInvalidValue;
  count_launch(total_spl > 0 ? 3 : 2);
  static std::atomic<int> occ[6] = {{0}, {0}, {0}, {0}, {0}, {0}};
  if (sc.key_level) {
    k_kmerge_init<<<(S + 127) / 128, 128, 0, stream>>>(sc.pairs, S, sc.half, sc.bounds, sc.ntiles);
    if (total_spl > 0) {
      k_kmerge_cuts<<<(total_spl + 7) / 8, 256, 0, stream>>>(sc.pairs, S, total_spl, sc.half,
                                                            sc.bounds);
    }
    if (sc.half == 512) {
      k_kmerge_tiles<512><<<merge_grid(k_kmerge_tiles<512>, occ[0], total_tiles), kThreads, 0,
                            stream>>>(sc.pairs, S, sc.bounds, sc.ntiles, sc.clook, sc.counter,
                                      total_tiles);
    } else if (sc.half == 1024) {
      k_kmerge_tiles<1024><<<merge_grid(k_kmerge_tiles<1024>, occ[1], total_tiles), kThreads, 0,
                             stream>>>(sc.pairs, S, sc.bounds, sc.ntiles, sc.clook, sc.counter,
                                       total_tiles);
    } else {
      k_kmerge_tiles<2048><<<merge_grid(k_kmerge_tiles<2048>, occ[2], total_tiles), kThreads, 0,
                             stream>>>(sc.pairs, S, sc.bounds, sc.ntiles, sc.clook, sc.counter,
                                       total_tiles);
    }
    return cudaGetLastError();
  }
  k_merge_init<<<(S + 127) / 128, 128, 0, stream>>>(sc.pairs, S, sc.half, sc.bounds, sc.ntiles);
  if (total_spl > 0) {
    k_merge_cuts<<<(total_spl + 7) / 8, 256, 0, stream>>>(sc.pairs, S, total_spl, sc.half,
                                                         sc.bounds);
  }
  if (sc.half == 512) {
    k_merge_tiles<512><<<merge_grid(k_merge_tiles<512>, occ[3], total_tiles), kThreads, 0,
                         stream>>>(sc.pairs, S, sc.bounds, sc.ntiles, sc.clook, sc.counter,
                                   total_tiles);
  } else if (sc.half == 1024) {
    k_merge_tiles<1024><<<merge_grid(k_merge_tiles<1024>, occ[4], total_tiles), kThreads, 0,
                          stream>>>(sc.pairs, S, sc.bounds, sc.ntiles, sc.clook, sc.counter,
                                    total_tiles);
  } else {
    k_merge_tiles<2048><<<merge_grid(k_merge_tiles<2048>, occ[5], total_tiles), kThreads, 0,
                          stream>>>(sc.pairs, S, sc.bounds, sc.ntiles, sc.clook, sc.counter,
                                    total_tiles);
  }
  return cudaGetLastError();
}

cudaError_t run_merge(const MergePair* h_pairs, int S, uint32_t total_spl, uint32_t total_tiles,
                      const MergeScratch& sc, cudaStream_t stream) {
  cudaError_t e = cudaMemcpyAsync(sc.pairs, h_pairs, sizeof(MergePair) * S,
                                  cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return e;
  MergeScratch s2 = sc;
  s2.key_level = S > 0;
  for (int i = 0; i < S; ++i) s2.key_level = s2.key_level && merge_key_level(h_pairs[i].a.bits);
  return run_merge_device(S, total_spl, total_tiles, s2, stream);
}

cudaError_t run_project_xy(const Levels& a, const Levels& out, cudaStream_t stream) {
  const uint64_t work = std::max<uint64_t>(a.cap1, 1);
  const unsigned blocks = (unsigned)std::min<uint64_t>((work + 255) / 256,
                                                       (uint64_t)device_sm_count() * 8);
  k_project_xy<<<blocks, 256, 0, stream>>>(a, out);
  count_launch(1);
  return cudaGetLastError();
}

size_t project_bitmap_scratch_bytes(uint32_t bits) {
  return align_up(((size_t)1 << (2 * bits)) / 8) + 2 * align_up(((size_t)1 << bits) * 4);
}

cudaError_t run_project_bitmap(const Levels& a, int plane, const Levels& out, void* scratch,
                               cudaStream_t stream) {
  const uint32_t b = a.bits;
  if (b < 5 || b > 13 || (plane != 1 && plane != 2)) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(scratch);
  uint32_t* bits = reinterpret_cast<uint32_t*>(p);
  const size_t bit_bytes = ((size_t)1 << (2 * b)) / 8;
  p += align_up(bit_bytes);
  uint32_t* rowcnt = reinterpret_cast<uint32_t*>(p);
  p += align_up(((size_t)1 << b) * 4);
  uint32_t* rowoff = reinterpret_cast<uint32_t*>(p);
  cudaError_t e = cudaMemsetAsync(bits, 0, bit_bytes, stream);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = (a.cap + kTile - 1) / kTile;
  if (tiles > 0) k_proj_set<<<(unsigned)tiles, kThreads, 0, stream>>>(a, plane, bits);
  const unsigned row_blocks = ((1u << b) + 7u) / 8u;  // a warp per row
  k_proj_rows<<<row_blocks, 256, 0, stream>>>(bits, b, rowcnt);
  k_proj_scan<<<1, kThreads, 0, stream>>>(rowcnt, b, rowoff, out, a.hdr);
  k_proj_write<<<row_blocks, 256, 0, stream>>>(bits, b, rowoff, out);
  count_launch(tiles > 0 ? 4 : 3);
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
