// Occupancy tree of a CGA for exact NN search (Eq. 7-8, Sec. V-C).
//
// The paper's window search bounds the search by the distance to the
// nearest x, y and z found so far.  For queries far from every stored voxel
// (a surface in a large box) that window still spans thousands of columns, so
// the search here also keeps a 64-ary tree of the occupied space: a node of
// level l is a cell of 4^l voxels per axis and records which of its 4 x 4 x 4
// sub-cells hold a voxel; level-1 nodes (bricks) record their 64 voxels.  A
// search descends nearest-first and skips every cell whose box lies farther
// than the best voxel found so far, so the result is still exactly Eq. 8's
// nearest voxel with the smaller-key rule.
//
// Build (all on the device, no host wait): the voxels are re-keyed by
// tree_key (each level's child number in 6 bits, coarsest level highest) by
// the sort pipeline's key pass, sorted by its radix passes, and every level
// is then one compaction of the sorted distinct prefixes of the level below
// (decoupled look-back over tiles for the output positions).
#include <algorithm>

#include "k_common.cuh"

namespace libcga {

namespace {

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

uint32_t tiles_of(uint64_t n) { return (uint32_t)std::max<uint64_t>(1, (n + kTile - 1) / kTile); }

// counts[0] = u of the CGA; counts[1..] = 0 (level sizes, set by the last
// tile of each level).
__global__ void k_tree_init(const Header* __restrict__ src, uint32_t* counts, uint32_t levels) {
  const uint32_t i = threadIdx.x;
  if (i <= levels) counts[i] = i == 0 ? (uint32_t)src->cnt[0] : 0u;
}

// One level of the tree from the sorted distinct prefixes P[0, n) of the
// level below (level 1: the voxels' tree keys): the distinct P >> 6 in order,
// each with its child set (bits P & 63) and the index in P of its first child.
// A tile of kTile prefixes is 256 threads x 16 consecutive entries.
// The box of a level-l node (l >= 2) comes from its children's boxes: a
// brick's (ccode1, voxel units) or a node's (cnode[.].w, in the child's
// grandchild units), each placed at its child position.
__global__ void __launch_bounds__(kThreads) k_tree_level(
    const unsigned long long* __restrict__ P, const uint32_t* n_in,
    unsigned long long* __restrict__ NP, unsigned long long* __restrict__ brick,
    uint32_t* __restrict__ bcode, uint4* __restrict__ node,
    const uint32_t* __restrict__ ccode1, const uint4* __restrict__ cnode,
    uint2* __restrict__ cpcode, uint32_t* n_out,
    uint32_t* look, uint32_t* counter, unsigned int* err) {
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_tile, s_excl;
  __shared__ unsigned long long s_k[kTile];
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint32_t n = *n_in;
  const uint32_t start = t * (uint32_t)kTile;
  if (start >= n) return;
  const uint32_t cnt = min((uint32_t)kTile, n - start);
  // the tile's prefixes staged by coalesced loads; each thread then takes 16
  // consecutive ones
  for (uint32_t e = tid; e < cnt; e += kThreads) s_k[e] = __ldg(P + start + e);
  __syncthreads();
  const uint32_t e0 = tid * kItems;
  unsigned long long k[kItems];
  uint32_t heads = 0;
  unsigned long long prev =
      e0 < cnt ? (e0 > 0 ? s_k[e0 - 1] : (start > 0 ? __ldg(P + start - 1) : 0ull)) : 0ull;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t e = e0 + i;
    k[i] = 0;
    if (e < cnt) {
      k[i] = s_k[e];
      if (start + e == 0 || (k[i] >> 6) != (prev >> 6)) heads |= 1u << i;
      prev = k[i];
    }
  }
  uint32_t tot = 0;
  const uint32_t off = block_excl_scan<uint32_t>((uint32_t)__popc(heads), tot, s_warp);
  if (tid == 0) {
    uint32_t excl = 0;
    st_relaxed(look + t, (t == 0 ? kFlagInc : kFlagAgg) | tot);
    if (t > 0) {
      excl = lookback(look, 1, t, 0, err);
      st_relaxed(look + t, kFlagInc | ((excl + tot) & kValMask));
    }
    s_excl = excl;
    if (start + cnt == n) *n_out = excl + tot;
  }
  __syncthreads();
  uint32_t j = s_excl + off;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (!((heads >> i) & 1u)) continue;
    const uint32_t e = start + e0 + i;
    const unsigned long long pr = k[i] >> 6;
    unsigned long long mask = 0;
    uint32_t lo[3] = {15u, 15u, 15u}, hi[3] = {0u, 0u, 0u};
    // a node has at most 64 children, so its run ends within 64 entries
    for (uint32_t f = e; f < n && f < e + 64; ++f) {
      const unsigned long long v = f == e ? k[i] : (f - start < cnt ? s_k[f - start] : __ldg(P + f));
      if ((v >> 6) != pr) break;
      const uint32_t c = (uint32_t)(v & 63);
      mask |= 1ull << c;
      if (brick == nullptr) {
        // the child's box in this node's grandchild units
        uint32_t pos[3];
        tree_cell(c, pos[0], pos[1], pos[2]);
        // the child's box in its own units: a brick's in voxels (0..3), a
        // node's in its grandchild cells (0..15)
        const uint32_t cc = ccode1 != nullptr ? __ldg(ccode1 + f) : __ldg(&cnode[f].w);
        const uint32_t m = ccode1 != nullptr ? 4u : 16u;  // child cell in those units
        uint32_t pl[3], ph[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const uint32_t cl = (cc >> (8 * a)) & 15u, ch = (cc >> (8 * a + 4)) & 15u;
          pl[a] = pos[a] * m + cl;
          ph[a] = pos[a] * m + ch;
          // in this node's grandchild cells (a node child's units are 4x finer)
          const uint32_t s = ccode1 != nullptr ? 0u : 2u;
          lo[a] = min(lo[a], pos[a] * 4 + (cl >> s));
          hi[a] = max(hi[a], pos[a] * 4 + (ch >> s));
        }
        cpcode[f] = make_uint2(pl[0] | ph[0] << 6 | pl[1] << 12 | ph[1] << 18, pl[2] | ph[2] << 6);
      }
    }
    if (NP != nullptr) NP[j] = pr;
    if (brick != nullptr) {
      brick[j] = mask;
      bcode[j] = tree_box_code(mask);
    } else {
      const uint32_t box = lo[0] | hi[0] << 4 | lo[1] << 8 | hi[1] << 12 | lo[2] << 16 | hi[2] << 20;
      node[j] = make_uint4((uint32_t)mask, (uint32_t)(mask >> 32), e, box);
    }
    ++j;
  }
}

// Words of the per-level look-back tables and tile counters (after the sort
// scratch).
size_t level_words(const TreeLayout& L) {
  size_t w = 0;
  for (uint32_t l = 1; l <= L.levels; ++l) w += tiles_of(L.cap[l - 1]) + 1;
  return w;
}

}  // namespace

TreeLayout tree_layout(uint32_t bits, uint64_t cap) {
  TreeLayout L{};
  L.levels = tree_levels(bits);
  L.cap[0] = cap;
  for (uint32_t l = 1; l <= L.levels; ++l) {
    const int cb = (int)bits - 2 * (int)l;  // bits of a level-l cell coordinate
    const uint64_t cells = cb <= 0 ? 1ull : (1ull << (3 * cb));
    L.cap[l] = std::min<uint64_t>(L.cap[l - 1], cells);
  }
  size_t p = 0;
  L.off[0] = p;  // error header + level counts
  p += align_up(sizeof(Header) + (kTreeMaxLevels + 1) * 4);
  L.off[1] = p;
  p += align_up(std::max<uint64_t>(L.cap[1], 1) * 8);
  L.off_bcode = p;
  p += align_up(std::max<uint64_t>(L.cap[1], 1) * 4);
  for (uint32_t l = 2; l <= L.levels; ++l) {
    L.off[l] = p;
    p += align_up(std::max<uint64_t>(L.cap[l], 1) * sizeof(uint4));
  }
  for (uint32_t l = 1; l < L.levels; ++l) {
    L.off_pcode[l] = p;
    p += align_up(std::max<uint64_t>(L.cap[l], 1) * sizeof(uint2));
  }
  L.bytes = p;
  return L;
}

TreeView tree_view(const TreeLayout& L, void* mem) {
  TreeView v{};
  char* b = static_cast<char*>(mem);
  v.brick = reinterpret_cast<const unsigned long long*>(b + L.off[1]);
  v.bcode = reinterpret_cast<const uint32_t*>(b + L.off_bcode);
  for (uint32_t l = 2; l <= L.levels; ++l) v.node[l] = reinterpret_cast<const uint4*>(b + L.off[l]);
  for (uint32_t l = 1; l < L.levels; ++l) v.pcode[l] = reinterpret_cast<const uint2*>(b + L.off_pcode[l]);
  for (uint32_t l = 1; l <= L.levels; ++l) v.cap[l] = (uint32_t)std::max<uint64_t>(L.cap[l], 1);
  v.levels = L.levels;
  return v;
}

size_t tree_scratch_bytes(const TreeLayout& L, uint32_t radix_bits) {
  const uint32_t tiles = tiles_of(L.cap[0]);
  return sort_scratch_bytes((uint64_t)tiles * kTile, tiles, 1, true, radix_bits) +
         align_up(level_words(L) * 4);
}

cudaError_t run_tree_build(const Levels& a, const TreeLayout& L, void* mem, void* scratch,
                           const Tuning& tu, unsigned int* err, cudaStream_t stream) {
  char* m = static_cast<char*>(mem);
  Header* hdr = reinterpret_cast<Header*>(m + L.off[0]);
  uint32_t* counts = reinterpret_cast<uint32_t*>(m + L.off[0] + sizeof(Header));
  const uint32_t tiles = tiles_of(L.cap[0]);
  const SortScratch sc =
      sort_scratch_carve(scratch, (uint64_t)tiles * kTile, tiles, 1, true, tu);
  uint32_t* lw = reinterpret_cast<uint32_t*>(
      static_cast<char*>(scratch) +
      sort_scratch_bytes((uint64_t)tiles * kTile, tiles, 1, true, tu.radix_bits));
  SortSeg seg{};
  seg.src = a;
  seg.plane = 4;
  seg.shift = L.levels;
  seg.from_cga = 1;
  seg.bits = a.bits;
  seg.key_bits = 6 * L.levels;
  seg.passes = radix_passes(seg.key_bits, tu.radix_bits);
  seg.bit0 = 0;
  seg.key_base = 0;
  seg.tile_base = 0;
  seg.num_tiles = tiles;
  // errors of the key pass and the radix passes' bounded waits land in the
  // CGA's own header (reported by its next cga_info)
  seg.out.hdr = a.hdr;
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(Header), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(lw, 0, level_words(L) * 4, stream);
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(sc.segs, &seg, sizeof(SortSeg), cudaMemcpyHostToDevice, stream);
  }
  if (e != cudaSuccess) return e;
  k_tree_init<<<1, kTreeMaxLevels + 1, 0, stream>>>(a.hdr, counts, L.levels);
  count_launch(1);
  if (L.cap[0] > 0) {
    e = run_sort_keys_device(1, tiles, seg.passes, sc, stream);
    if (e != cudaSuccess) return e;
  }
  unsigned long long* buf[2] = {static_cast<unsigned long long*>(sc.keys0),
                                static_cast<unsigned long long*>(sc.keys1)};
  int cur = (int)(seg.passes & 1u);  // the buffer holding the sorted keys
  unsigned int* herr = err != nullptr ? err : &hdr->err;
  uint32_t* w = lw;
  for (uint32_t l = 1; l <= L.levels && L.cap[0] > 0; ++l) {
    const uint32_t lt = tiles_of(L.cap[l - 1]);
    unsigned long long* np = l < L.levels ? buf[cur ^ 1] : nullptr;
    unsigned long long* br = l == 1 ? reinterpret_cast<unsigned long long*>(m + L.off[1]) : nullptr;
    uint32_t* bc = l == 1 ? reinterpret_cast<uint32_t*>(m + L.off_bcode) : nullptr;
    uint4* nd = l >= 2 ? reinterpret_cast<uint4*>(m + L.off[l]) : nullptr;
    const uint32_t* cc1 = l == 2 ? reinterpret_cast<const uint32_t*>(m + L.off_bcode) : nullptr;
    const uint4* cn = l >= 3 ? reinterpret_cast<const uint4*>(m + L.off[l - 1]) : nullptr;
    uint2* cp = l >= 2 ? reinterpret_cast<uint2*>(m + L.off_pcode[l - 1]) : nullptr;
    k_tree_level<<<lt, kThreads, 0, stream>>>(buf[cur], counts + (l - 1), np, br, bc, nd, cc1, cn,
                                             cp, counts + l, w, w + lt, herr);
    count_launch(1);
    w += lt + 1;
    cur ^= 1;
  }
  return cudaGetLastError();
}

}  // namespace libcga
