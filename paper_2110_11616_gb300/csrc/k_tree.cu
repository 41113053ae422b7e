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
  // Each item is a child of the node its prefix >> 6 names: its contribution
  // (its bit in the child set and, above the bricks, its box in the node's
  // grandchild cells, as bytes lo_x | lo_y << 8 | lo_z << 16 and the same for
  // hi) is formed item by item, and runs of one node are reduced within the
  // thread, then across threads by a reverse segmented scan: a node's record
  // is written by the thread holding its first child once its run is whole.
  // Only the tile's last run can go on into the next tile: its head thread
  // reads the rest (at most 63 children) from global memory.
  const bool nodes = brick == nullptr;
  auto contrib = [&](uint32_t f, unsigned long long v, uint32_t& lo, uint32_t& hi) {
    lo = 0x0F0F0Fu;
    hi = 0u;
    if (!nodes) return;
    const uint32_t c = (uint32_t)(v & 63);
    uint32_t pos[3];
    tree_cell(c, pos[0], pos[1], pos[2]);
    // the child's box in its own units: a brick's in voxels (0..3), a node's
    // in its grandchild cells (0..15)
    const uint32_t cc = ccode1 != nullptr ? __ldg(ccode1 + f) : __ldg(&cnode[f].w);
    const uint32_t m = ccode1 != nullptr ? 4u : 16u;  // child cell in those units
    const uint32_t s = ccode1 != nullptr ? 0u : 2u;   // a node child's units are 4x finer
    uint32_t pl[3], ph[3];
    lo = 0u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const uint32_t cl = (cc >> (8 * a)) & 15u, ch = (cc >> (8 * a + 4)) & 15u;
      pl[a] = pos[a] * m + cl;
      ph[a] = pos[a] * m + ch;
      lo |= (pos[a] * 4 + (cl >> s)) << (8 * a);
      hi |= (pos[a] * 4 + (ch >> s)) << (8 * a);
    }
    cpcode[f] = make_uint2(pl[0] | ph[0] << 6 | pl[1] << 12 | ph[1] << 18, pl[2] | ph[2] << 6);
  };
  auto write_node = [&](uint32_t jj, uint32_t first, unsigned long long pr,
                        unsigned long long mask, uint32_t lo, uint32_t hi) {
    if (NP != nullptr) NP[jj] = pr;
    if (!nodes) {
      brick[jj] = mask;
      bcode[jj] = tree_box_code(mask);
    } else {
      uint32_t box = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        box |= (((lo >> (8 * a)) & 15u) | ((hi >> (8 * a)) & 15u) << 4) << (8 * a);
      }
      node[jj] = make_uint4((uint32_t)mask, (uint32_t)(mask >> 32), first, box);
    }
  };
  uint32_t j = s_excl + off;
  // the thread's own items: the leading part (before its first head) and
  // the run of its last head so far
  unsigned long long am = 0, lead_m = 0, hpr = 0;  // hpr: the current head's node
  uint32_t alo = 0x0F0F0Fu, ahi = 0u, lead_lo = 0x0F0F0Fu, lead_hi = 0u, hfirst = 0;
  int head_i = -1;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t e = e0 + i;
    if (e >= cnt) break;
    uint32_t clo, chi;
    contrib(start + e, k[i], clo, chi);
    if ((heads >> i) & 1u) {
      if (head_i < 0) {
        lead_m = am;
        lead_lo = alo;
        lead_hi = ahi;
      } else {
        // the previous head's run ends inside the thread
        write_node(j, hfirst, hpr, am, alo, ahi);
        ++j;
      }
      head_i = i;
      hpr = k[i] >> 6;
      hfirst = start + e;
      am = 0;
      alo = 0x0F0F0Fu;
      ahi = 0u;
    }
    am |= 1ull << (k[i] & 63);
    alo = __vminu4(alo, clo);
    ahi = __vmaxu4(ahi, chi);
  }
  if (head_i < 0) {
    lead_m = am;
    lead_lo = alo;
    lead_hi = ahi;
  }
  // reverse segmented scan over the threads of the leading parts: thread u
  // ends with the union of the leading parts of threads u, u + 1, ... up to
  // and including the first thread that holds a head
  const uint32_t lane = tid & 31u, w = tid >> 5;
  unsigned long long sm = lead_m;
  uint32_t slo = lead_lo, shi = lead_hi;
  bool sf = head_i >= 0;
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const unsigned long long om = __shfl_down_sync(0xffffffffu, sm, d);
    const uint32_t olo = __shfl_down_sync(0xffffffffu, slo, d);
    const uint32_t ohi = __shfl_down_sync(0xffffffffu, shi, d);
    const bool of = __shfl_down_sync(0xffffffffu, sf, d);
    if (lane + d < 32 && !sf) {
      sm |= om;
      slo = __vminu4(slo, olo);
      shi = __vmaxu4(shi, ohi);
      sf = of;
    }
  }
  __shared__ unsigned long long s_wm[kWarps], s_tm[kThreads];
  __shared__ uint32_t s_wlo[kWarps], s_whi[kWarps], s_tlo[kThreads], s_thi[kThreads];
  __shared__ uint8_t s_wf[kWarps], s_tf[kThreads];
  if (lane == 0) {
    s_wm[w] = sm;
    s_wlo[w] = slo;
    s_whi[w] = shi;
    s_wf[w] = sf ? 1 : 0;
  }
  __syncthreads();
  for (uint32_t x = w + 1; x < (uint32_t)kWarps && !sf; ++x) {
    sm |= s_wm[x];
    slo = __vminu4(slo, s_wlo[x]);
    shi = __vmaxu4(shi, s_whi[x]);
    sf = s_wf[x] != 0;
  }
  s_tm[tid] = sm;
  s_tlo[tid] = slo;
  s_thi[tid] = shi;
  s_tf[tid] = sf ? 1 : 0;
  __syncthreads();
  if (head_i >= 0) {
    // the last head's run: the thread's tail, the leading parts that follow
    bool closed = false;
    if (tid + 1 < (uint32_t)kThreads) {
      am |= s_tm[tid + 1];
      alo = __vminu4(alo, s_tlo[tid + 1]);
      ahi = __vmaxu4(ahi, s_thi[tid + 1]);
      closed = s_tf[tid + 1] != 0;
    }
    if (!closed) {
      // the run reaches the end of the tile: the rest lies in the next one
      for (uint32_t f = start + cnt; f < n && f < start + cnt + 64; ++f) {
        const unsigned long long v = __ldg(P + f);
        if ((v >> 6) != hpr) break;
        am |= 1ull << (v & 63);
        if (nodes) {
          // (the next tile writes this child's own box in the parent frame)
          const uint32_t c = (uint32_t)(v & 63);
          uint32_t pos[3];
          tree_cell(c, pos[0], pos[1], pos[2]);
          const uint32_t cc = ccode1 != nullptr ? __ldg(ccode1 + f) : __ldg(&cnode[f].w);
          const uint32_t s = ccode1 != nullptr ? 0u : 2u;
          uint32_t clo = 0, chi = 0;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            clo |= (pos[a] * 4 + (((cc >> (8 * a)) & 15u) >> s)) << (8 * a);
            chi |= (pos[a] * 4 + (((cc >> (8 * a + 4)) & 15u) >> s)) << (8 * a);
          }
          alo = __vminu4(alo, clo);
          ahi = __vmaxu4(ahi, chi);
        }
      }
    }
    write_node(j, hfirst, hpr, am, alo, ahi);
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
