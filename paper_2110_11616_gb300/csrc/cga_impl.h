// Internal structures shared by the libcga kernels and the C-ABI layer.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace libcga {

// Tiling shared by the sort pipeline: 256 threads x 16 keys per tile.
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096
constexpr int kRadixBits = 8;  // default digit width (and the NN query sort's)
constexpr int kRadix = 1 << kRadixBits;
constexpr int kRadixMaxBits = 9;
constexpr int kMaxPasses = 6;  // 3 * 16 bits / 8 (or / 9)

// Launch shape of the sort and merge kernels, chosen per (grid bits, size
// bucket) by measurement (cga_autotune) and held in a process-wide table.
struct Tuning {
  uint32_t radix_bits;    // digit width of an LSD pass: 8 or 9
  uint32_t sort_threads;  // threads per 4096-key tile: 256 (16 keys each) or 512 (8 keys each)
  uint32_t merge_half;    // merge-path partition: a splitter every merge_half points (512..2048)
};
constexpr Tuning kDefaultTuning{8u, 512u, 2048u};
bool tuning_valid(const Tuning& t);
// The table entry for grids of `bits` per axis and n elements (the default
// when none was set).  Host only, thread-safe.
Tuning tuning_for(uint32_t bits, uint64_t n);
void tuning_store(uint32_t bits, uint64_t n, const Tuning* t);  // nullptr: back to the default
inline uint32_t radix_passes(uint32_t key_bits, uint32_t radix_bits) {
  return (key_bits + radix_bits - 1) / radix_bits;
}

// Device error bits recorded in a handle header.
enum : uint32_t { kErrNonfinite = 1u, kErrTimeout = 2u };

// Counts of a compacted level structure.  For a 3-level CGA cnt = {u, g, h};
// for a 2-level projection cnt = {g2 (|V|), h2 (|U|), 0}.
struct alignas(16) Header {
  unsigned long long cnt[3];
  unsigned int err;
  unsigned int pad;
};

// Output (or input) arrays of a CGA.  Level 0 is the finest (Z_index, or
// V_index of a projection); level 1 is Y (or U) with its pointer array;
// level 2 is X (absent in a projection).
struct Levels {
  uint16_t* idx0;
  uint16_t* idx1;
  uint32_t* ptr1;
  uint16_t* idx2;
  uint32_t* ptr2;
  Header* hdr;
  uint32_t bits;
  uint32_t nlevels;  // 3 or 2
  uint64_t cap;      // capacity of level 0 (>= u)
  uint64_t cap1;     // capacity of level 1
  uint64_t cap2;     // capacity of level 2 (0 for a projection)
};

// One segment (cloud) of the sort pipeline.
struct SortSeg {
  // build input (nullptr for a projection)
  const float* xyz;
  float scale;
  float off[3];
  float X[12];
  uint32_t has_x;
  // projection input: the source CGA and the plane
  Levels src;
  int32_t plane;      // 0 xy, 1 xz, 2 yz: 2D re-key; 3: coarsen (3D, >> shift);
                      // 4: occupancy-tree key (tree_key of x, y, z over `shift` levels)
  uint32_t shift;     // plane 3: coarse cell = 2^shift voxels per axis; plane 4: levels
  uint32_t from_cga;  // 1: keys come from src (projection), 0: from xyz
  // common
  uint32_t n_host;      // element count when known on the host (build)
  uint32_t bits;        // grid bits of this segment
  uint32_t key_bits;    // significant key bits: 3b (build) or 2b (projection)
  uint32_t passes;      // radix passes = ceil(key_bits / radix_bits)
  uint32_t bit0;        // lowest key bit sorted on (pass p sorts bits bit0 + p * radix_bits ..)
  uint64_t key_base;    // first key slot of this segment in the key buffers
  uint32_t tile_base;   // first global tile index
  uint32_t num_tiles;   // tiles reserved (from the capacity)
  Levels out;           // compacted output
};

// Scratch layout of one sort-pipeline run (all offsets from one base).
struct SortScratch {
  void* keys0;
  void* keys1;
  uint32_t* hist;      // [S][kMaxPasses][2^radix_bits]
  uint32_t* look;      // [kMaxPasses][total_tiles][2^radix_bits]
  uint32_t* clook;     // [total_tiles][3]
  uint32_t* counters;  // [kMaxPasses + 1]
  SortSeg* segs;       // [S]
  size_t zero_bytes;   // bytes from hist to the end of counters
  uint32_t radix_bits;    // launch shape of the passes (Tuning)
  uint32_t sort_threads;
};

// Scratch of a sort run; the digit width sizes the histogram and look-back
// tables, the thread count only selects the pass kernel.
size_t sort_scratch_bytes(uint64_t total_keys, uint32_t total_tiles, int S, bool key64,
                          uint32_t radix_bits = kRadixBits);
SortScratch sort_scratch_carve(void* base, uint64_t total_keys, uint32_t total_tiles, int S,
                               bool key64, const Tuning& tu = kDefaultTuning);
// Set the shared-memory limits of the pass kernels (once; before any graph
// capture that launches them).
cudaError_t init_sort_kernels();
// Query the residency of the NN search kernels (once; before any capture).
void init_nn_kernels();

// Queue only the radix passes (segments already on the device in sc.segs,
// histograms filled, look-back words zeroed).
cudaError_t run_radix_passes(int S, uint32_t total_tiles, uint32_t max_passes, bool key64,
                             const SortScratch& sc, cudaStream_t stream);

// Only key generation and the radix passes of 64-bit keys (segment table on
// the device; no compaction): the sorted keys end in keys0 after an even
// number of passes, in keys1 after an odd one.
cudaError_t run_sort_keys_device(int S, uint32_t total_tiles, uint32_t max_passes,
                                 const SortScratch& sc, cudaStream_t stream);

// Sort pipeline with the segment table already on the device (sc.segs).
cudaError_t run_sort_device(int S, uint32_t total_tiles, uint32_t max_passes, bool key64,
                            int levels, const SortScratch& sc, cudaStream_t stream);

// Queue the whole sort pipeline: header init, key generation (+ histograms),
// radix passes, compaction.  `h_segs` is copied to the device first.
cudaError_t run_sort_pipeline(const SortSeg* h_segs, int S, uint32_t total_tiles,
                              uint32_t max_passes, bool key64, const SortScratch& sc,
                              cudaStream_t stream);

// ---- operations on built CGAs ---------------------------------------------

// Decode a CGA to uint32 (x, y, z) triples in CGA order.
cudaError_t run_decode(const Levels& a, uint32_t* xyz, cudaStream_t stream);

// Merge: sorted union of pairs of 3-level CGAs, column by column (or, on fine
// grids, key by key).  Splitters are taken at every half-th (x, y) column
// (or point) of each input (half = Tuning::merge_half <= kTile / 2; `cap`
// below is a point capacity, which bounds the columns too); between
// consecutive splitters each input contributes at most half columns (points),
// so one tile of at most 2 * half of them always holds the merged run.
constexpr int kMergeHalf = kTile / 2;  // largest partition
inline uint32_t merge_splitters(uint64_t cap, uint32_t half) {
  return cap > 0 ? (uint32_t)((cap - 1) / half) : 0u;
}

struct MergePair {
  Levels a, b, out;
  uint32_t spl_base;   // splitter slots: A's [spl_base, +spl_a), then B's spl_b
  uint32_t spl_a, spl_b;
  uint32_t tile_base;  // reserved tiles: spl_a + spl_b + 1
  uint32_t num_tiles;
};

struct MergeScratch {
  uint32_t* bounds;         // [(total_tiles + S) * 4]; pair p at 4 * (tile_base + p)
  uint32_t* ntiles;         // [S]
  uint32_t* clook;          // [total_tiles][3]
  uint32_t* counter;        // [1]
  MergePair* pairs;         // [S]
  size_t zero_bytes;        // clook .. counter
  uint32_t half;            // merge-path partition the splitters were counted with
  bool key_level;           // merge the key sequences instead of the columns
};
// The merge form for pairs on grids of `bits` per axis: key-level from 14 bits
// on (a column then holds about one voxel), column-level below.
inline bool merge_key_level(uint32_t bits) { return bits >= 14; }

size_t merge_scratch_bytes(uint32_t total_spl, uint32_t total_tiles, int S);
MergeScratch merge_scratch_carve(void* base, uint32_t total_spl, uint32_t total_tiles, int S,
                                 uint32_t half = kMergeHalf);
cudaError_t run_merge(const MergePair* h_pairs, int S, uint32_t total_spl, uint32_t total_tiles,
                      const MergeScratch& sc, cudaStream_t stream);
// Merge with the pair table already on the device (sc.pairs).
cudaError_t run_merge_device(int S, uint32_t total_spl, uint32_t total_tiles,
                             const MergeScratch& sc, cudaStream_t stream);

// ---- Value array (Sec. V) -----------------------------------------------
constexpr int kValueAverage = 0;  // a voxel's row: round-half-up mean of its points
constexpr int kValueFirst = 1;    // a voxel's row: its first input point's
constexpr int kMergeBase = 0;     // a voxel in both merge inputs keeps the base's row
constexpr int kMergeAverage = 1;  // or (a + b + 1) / 2 per channel

// The points and attributes a build's Value array is made from, with the
// build's grid and transform (the same voxel keys as the build).
struct ValueInput {
  const float* xyz;
  const uint8_t* attr;  // n * channels, point order
  uint64_t n;
  uint32_t channels;    // 1..4
  int policy;           // kValueAverage or kValueFirst
  float scale;
  float off[3];
  float X[12];
  uint32_t has_x;
};
size_t value_scratch_bytes(uint64_t cap, uint32_t channels, int policy);
// values (a.cap * channels bytes) for the CGA a built from in (queued after
// the build on the same stream); scratch of value_scratch_bytes.
cudaError_t run_build_values(const Levels& a, const ValueInput& in, void* scratch,
                             uint8_t* values, cudaStream_t stream);
// vm (m.cap * channels bytes) for m = merge(a, b) with rows va, vb.
cudaError_t run_merge_values(const Levels& m, const Levels& a, const Levels& b, const uint8_t* va,
                             const uint8_t* vb, uint32_t channels, int policy, uint8_t* vm,
                             cudaStream_t stream);

// ---- Radius search and k-NN ------------------------------------------------
// One CGA and its queries (grid as the CGA's).
struct SearchSeg {
  Levels a;
  float scale;
  float off[3];
  const float* q;  // m points, float32 AoS
  uint32_t m;
  const uint4* ctab;  // the NN column table of `a` (cga_nn_prepare) or null
};
size_t radius_scratch_bytes();
// order (or null): the queries' Morton keys of the NN search (query index in
// the low 32 bits), visited in that order.
// offsets (m + 1): exclusive prefix of the per-query counts, offsets[m] = total.
cudaError_t run_radius_count(const SearchSeg& sg, unsigned long long r2,
                             const unsigned long long* order, unsigned long long* offsets,
                             void* scratch, cudaStream_t stream);
cudaError_t run_radius_fill(const SearchSeg& sg, unsigned long long r2,
                            const unsigned long long* order, const unsigned long long* offsets,
                            uint32_t* idx, unsigned long long* d2, cudaStream_t stream);
// idx, d2: m * k entries (k <= kKnnMaxK), query j's k nearest ascending.
constexpr uint32_t kKnnMaxK = 1024;
cudaError_t run_knn(const SearchSeg& sg, uint32_t k, const unsigned long long* order, uint32_t* idx,
                    unsigned long long* d2, cudaStream_t stream);

// ---- Perspective projection (Eq. 5-6) ---------------------------------------
struct Camera {
  float eye[3];         // voxel units
  float cos_t, sin_t;   // rotation about the y axis
  float D;              // distance of the projection plane
  uint32_t W, H;        // image size in pixels
};
// index / depth: W * H pixels; zbuf: W * H 64-bit words of scratch.
cudaError_t run_perspective(const Levels& a, const Camera& cam, unsigned long long* zbuf,
                            uint32_t* index, float* depth, cudaStream_t stream);

// ---- Compression pieces (Sec. V-D) and the G-Arrays X pointer ----------------
constexpr uint32_t kKmClusters = 8;  // one centre per corner of the bounding box
// Device state of one k-means run.
struct KmState {
  unsigned long long sum[kKmClusters][4];  // x, y, z sums and count of a pass
  unsigned long long changed;              // labels a pass changed
  uint32_t box[6];                         // least y, z (box[1..2]), greatest (box[4..5])
  uint32_t pass, done, max_iter;
};
// labels: u bytes; centres: 8 * 3 in 1/256 voxel; counts: 8; iters: 1.
cudaError_t run_kmeans(const Levels& a, uint32_t max_iter, KmState* st, uint8_t* labels,
                       long long* centres, unsigned long long* counts, uint32_t* iters,
                       cudaStream_t stream);
cudaError_t run_motion(const long long* ref_c, const unsigned long long* ref_n,
                       const long long* pred_c, const unsigned long long* pred_n, long long* mv,
                       cudaStream_t stream);
// out: u * 3 int32 voxels.
cudaError_t run_reconstruct(const Levels& a, const uint8_t* labels, const long long* mv, int* out,
                            cudaStream_t stream);
// res: u_pred * channels int16.
cudaError_t run_residual(const uint8_t* pred, uint64_t u_pred, const uint8_t* ref, uint64_t u_ref,
                         const uint32_t* idx, uint32_t channels, int16_t* res,
                         cudaStream_t stream);
// xptr: 2^bits + 1 entries.
cudaError_t run_garrays_x(const Levels& a, uint32_t* xptr, cudaStream_t stream);
// xptr == nullptr: the CGA lookup; else through the dense X pointer.
cudaError_t run_lookup(const Levels& a, const uint32_t* xptr, const int* qv, uint32_t m,
                       uint32_t* idx, cudaStream_t stream);

// Copy the top two levels of a CGA into a 2-level projection (plane xy).
cudaError_t run_project_xy(const Levels& a, const Levels& out, cudaStream_t stream);
// The xz (plane 1) or yz (plane 2) projection of a CGA on a grid of 5 to 13
// bits per axis through a bitmap of its 2D voxels (no sort); scratch of
// project_bitmap_scratch_bytes(bits).
constexpr uint32_t kProjBitmapMinBits = 5, kProjBitmapMaxBits = 13;
size_t project_bitmap_scratch_bytes(uint32_t bits);
cudaError_t run_project_bitmap(const Levels& a, int plane, const Levels& out, void* scratch,
                               cudaStream_t stream);
struct ProjPair {
  Levels a, out;
};
// S xy projections in one launch (pair table on the device).
cudaError_t run_project_xy_device(const ProjPair* d_pairs, int S, uint64_t max_cap1,
                                  cudaStream_t stream);

// Exact NN: one segment per (CGA, query batch).  Queries occupy a slot space
// of whole tiles (segment s owns slots [tile_base*kTile, (tile_base +
// num_tiles)*kTile)).  With scratch the queries are first sorted along a
// Morton curve so that neighbouring warps search neighbouring space.
constexpr int kMaxCoarse = 2;

// Occupancy tree of a CGA for NN search (cga_nn_prepare_levels with
// CGA_NN_TREE): a 64-ary tree over the grid in which a node of level l covers
// 4^l voxels per axis and has up to 4 x 4 x 4 children of level l - 1,
// numbered by tree_child (bit p of a node's child set is its child number p).
// Level 1 nodes (bricks) hold their 64 voxels as occupancy bits, numbered the
// same way; the root is level tree_levels(bits), with node 0 of that level
// the only one.
constexpr int kTreeMaxLevels = 8;  // ceil(16 / 2)
inline uint32_t tree_levels(uint32_t bits) { return (bits + 1) / 2; }
// Number of the child cell (cx, cy, cz) in [0, 4)^3 of a tree cell:
// p = s << 4 | t << 2 | cx with s = (cx + cy) mod 4 and t = (cy + cz) mod 4.
// Any plane of cells with one coordinate fixed holds one cell of each
// (s, t), so a search that gives each lane the children of a fixed range of
// numbers (4, 8 or 16 consecutive ones) sees the 16 children of such a plane
// split evenly over its lanes.  Voxels inside a brick are numbered the same
// way.
__host__ __device__ inline uint32_t tree_child(uint32_t cx, uint32_t cy, uint32_t cz) {
  return ((cx + cy) & 3u) << 4 | ((cy + cz) & 3u) << 2 | cx;
}
// The cell of child number p (the inverse of tree_child).
__host__ __device__ inline void tree_cell(uint32_t p, uint32_t& cx, uint32_t& cy, uint32_t& cz) {
  cx = p & 3u;
  cy = ((p >> 4) - cx) & 3u;
  cz = (((p >> 2) & 3u) - cy) & 3u;
}
// Key of voxel (x, y, z) in the tree's order: bits [6(l-1), 6l) hold the
// child number (tree_child) of the voxel's level-(l-1) cell inside its
// level-l cell, for l = 1..levels.  Ascending keys list the voxels brick by
// brick in a depth-first walk of the tree.
__host__ __device__ inline unsigned long long tree_key(uint32_t x, uint32_t y, uint32_t z,
                                                       uint32_t levels) {
  unsigned long long k = 0;
  for (uint32_t l = 0; l < levels; ++l) {
    const uint32_t c = tree_child((x >> (2 * l)) & 3u, (y >> (2 * l)) & 3u, (z >> (2 * l)) & 3u);
    k |= (unsigned long long)c << (6 * l);
  }
  return k;
}
// The child numbers whose cell has coordinate v on axis a: bit p of
// tree_axis_set(a, v) is set when tree_cell(p) puts p at v on that axis.
__host__ __device__ constexpr unsigned long long tree_axis_set(int a, uint32_t v) {
  unsigned long long m = 0;
  for (uint32_t p = 0; p < 64; ++p) {
    const uint32_t cx = p & 3u, cy = ((p >> 4) - cx) & 3u, cz = (((p >> 2) & 3u) - cy) & 3u;
    if ((a == 0 ? cx : (a == 1 ? cy : cz)) == v) m |= 1ull << p;
  }
  return m;
}
// Box of a brick's occupied voxels from its voxel set m (m != 0; bit p =
// tree_child of the voxel inside the brick), in voxels (0..3 per axis):
// lo_x | hi_x << 4 | lo_y << 8 | hi_y << 12 | lo_z << 16 | hi_z << 20 (the
// field layout of a node's box).  Per axis the occupied coordinates are the
// coordinate sets m meets; their least and greatest are the bounds.
template <int A>
__host__ __device__ inline uint32_t tree_axis_bounds(unsigned long long m) {
  // (constants: the four coordinate sets of axis A)
  constexpr unsigned long long s0 = tree_axis_set(A, 0), s1 = tree_axis_set(A, 1),
                               s2 = tree_axis_set(A, 2), s3 = tree_axis_set(A, 3);
  const uint32_t occ = ((m & s0) ? 1u : 0u) | ((m & s1) ? 2u : 0u) | ((m & s2) ? 4u : 0u) |
                       ((m & s3) ? 8u : 0u);
  const uint32_t lo = occ & 1u ? 0u : (occ & 2u ? 1u : (occ & 4u ? 2u : 3u));
  const uint32_t hi = occ & 8u ? 3u : (occ & 4u ? 2u : (occ & 2u ? 1u : 0u));
  return lo | hi << 4;
}
__host__ __device__ inline uint32_t tree_box_code(unsigned long long m) {
  return tree_axis_bounds<0>(m) | tree_axis_bounds<1>(m) << 8 | tree_axis_bounds<2>(m) << 16;
}
// A node of level l >= 2 keeps the box of its occupied voxels at the
// granularity of its grandchildren (cells of 4^(l-2) voxels; 16 per axis of
// the node): lo_x | hi_x << 4 | lo_y << 8 | hi_y << 12 | lo_z << 16 | hi_z << 20.
// Every entry of a level l below the root also keeps its box in its parent's
// frame (pcode): 6-bit bounds counted from the parent's origin in cells of
// 4^(l-2) voxels (l >= 2) or in voxels (bricks), Lx | Hx << 6 | Ly << 12 |
// Hy << 18 in .x and Lz | Hz << 6 in .y; the box along x covers
// [Lx * u, (Hx + 1) * u) voxels from the parent's origin for that unit u.
struct TreeView {
  const unsigned long long* brick;        // level 1: voxel occupancy of each brick
  const uint32_t* bcode;                  // level 1: tree_box_code of each brick (voxel units)
  const uint4* node[kTreeMaxLevels + 1];  // level l >= 2: {child set lo, hi, first child,
                                          //  box of the voxels in grandchild units}
  const uint2* pcode[kTreeMaxLevels + 1]; // level l < levels: box in the parent's frame
  uint32_t cap[kTreeMaxLevels + 1];       // entries reserved per level (a search never reads beyond)
  uint32_t levels;                        // 0: no tree
};
// Capacity of every level (cap[0]: voxels) and the bytes of the tree arrays
// (offsets from one base: off[1] bricks, off_bcode their box codes, off[l]
// nodes of level l, off_pcode[l] the boxes of level l in their parents'
// frames, off[0] the device counts, one 32-bit word per level).
struct TreeLayout {
  uint64_t cap[kTreeMaxLevels + 1];
  size_t off[kTreeMaxLevels + 1];
  size_t off_pcode[kTreeMaxLevels + 1];
  size_t off_bcode;
  size_t bytes;
  uint32_t levels;
};
TreeLayout tree_layout(uint32_t bits, uint64_t cap);
// Scratch of one tree build (the Morton-key sort and the per-level
// look-back words).
size_t tree_scratch_bytes(const TreeLayout& L, uint32_t radix_bits);
// Build the tree of a into mem (laid out by L): Morton keys of the voxels,
// sorted by radix passes, then one compaction per level from the bricks up.
// Errors of a bounded wait are recorded in err.
cudaError_t run_tree_build(const Levels& a, const TreeLayout& L, void* mem, void* scratch,
                           const Tuning& tu, unsigned int* err, cudaStream_t stream);
TreeView tree_view(const TreeLayout& L, void* mem);

struct NnSeg {
  Levels a;
  // optional coarse levels (ncoarse = 0..kMaxCoarse, coarsest last): c[k] is
  // the CGA of the occupied cells of 2^shift[k] voxels per axis, xs[k][j] the
  // first slab of the next finer level inside c[k]'s slab j (one past the last
  // slab = that level's slab count), cxdir[k] c[k]'s x directory (or null)
  Levels c[kMaxCoarse];
  const uint32_t* xs[kMaxCoarse];
  uint32_t shift[kMaxCoarse];
  const uint32_t* cxdir[kMaxCoarse];
  // zr[k][c] = {first cell, end, lowest | highest << 16 cell z, 0} of column c
  // of c[k] (or null): the column table of the level
  const uint4* zr[kMaxCoarse];
  // child[k][(c << dsh) + j]: for column c of c[k] (dsh = its shift minus the
  // next finer level's), the first column of the j-th finer slab under it
  // with y >= its y << dsh (or null: found by a search instead)
  const uint32_t* child[kMaxCoarse];
  uint32_t ncoarse;
  // optional x directory of `a` (cga_nn_prepare): for every x value v of the
  // grid, the index of the first X_index entry >= v
  const uint32_t* xdir;
  // optional column table of `a` (cga_nn_prepare): per column {first voxel,
  // end, lowest z | highest z << 16, 0}
  const uint4* ctab;
  // optional occupancy tree of `a`; when present the tree search runs
  TreeView tree;
  float scale;
  float off[3];
  const float* q;
  // integer query voxels (m * 3) instead of q when not null
  const int* qv;
  uint32_t m;
  uint32_t* idx;
  unsigned long long* d2;
  uint32_t tile_base;
  uint32_t num_tiles;
};
constexpr uint64_t kNnSortMin = 8192;
constexpr uint64_t kNnMaxQueries = (1u << 30) - 1u;  // per segment
size_t nn_scratch_bytes(uint32_t total_tiles, int S);
// scratch == nullptr: no query sort, S must be 1 (the segment travels as a
// kernel parameter).
cudaError_t run_nn(const NnSeg* h_segs, int S, uint32_t total_tiles, void* scratch,
                   cudaStream_t stream);
// Device-side tables of an NN batch carved from its scratch.
struct NnTables {
  Header* err;
  NnSeg* segs;
  SortScratch sort;
};
NnTables nn_tables(void* scratch, uint32_t total_tiles, int S);
// Upload the NnSeg and sort-segment tables (pageable copies, not capturable).
cudaError_t nn_upload(const NnSeg* h_segs, int S, const NnTables& t, cudaStream_t stream);
// Upload the tables of one segment from stack copies (no heap allocation).
cudaError_t nn_upload_one(const NnSeg& h_seg, const NnTables& t, cudaStream_t stream);
// Only the query sort (keys in t.sort.keys0 afterwards), or only the search of
// one segment with a given order (nullptr: query order).
cudaError_t run_nn_sort_device(int S, uint32_t total_tiles, const NnTables& t,
                               cudaStream_t stream);
cudaError_t run_nn_search(const NnSeg& seg, const unsigned long long* order, cudaStream_t stream);
// Search kernel a segment needs: 0 the fine search, 1 or 2 the coarse
// levels, 3 the occupancy tree.
inline uint32_t nn_kind(const NnSeg& s) { return s.tree.levels > 0 ? 3u : s.ncoarse; }
// Run with the tables on the device (capturable: memsets and kernels only).
// kinds: bit k set when some segment has nn_kind k (selects the kernels: the
// tree search for segments with a tree, the window search of the largest
// other kind for the rest).
cudaError_t run_nn_device(int S, uint32_t total_tiles, const NnTables& t, cudaStream_t stream,
                          uint32_t kinds = 1u);

// For each slab k of the coarse CGA c (cells of 2^shift voxels), xs[k] = first
// index of a's X_index whose x >> shift equals c's X_index[k]; xs[h_c] = h_a.
cudaError_t run_coarse_slab_index(const Levels& a, const Levels& c, uint32_t shift, uint32_t* xs,
                                  cudaStream_t stream);

// For every column of the coarse level c (dsh bits coarser than f, xs its
// slab index into f): the first column of each finer slab under it at or
// above its y range.  child has c.cap1 << dsh entries.
cudaError_t run_child_columns(const Levels& f, const Levels& c, const uint32_t* xs, uint32_t dsh,
                              uint32_t* child, cudaStream_t stream);
// t[c] = {Y_pointer[c], Y_pointer[c + 1], Z_index[Y_pointer[c]] |
// Z_index[Y_pointer[c + 1] - 1] << 16, 0} for every column c of a (a.cap1
// entries reserved).
cudaError_t run_column_table(const Levels& a, uint4* t, cudaStream_t stream);
// xdir[v] = first index of a's X_index with value >= v, for v in [0, 2^bits].
cudaError_t run_x_directory(const Levels& a, uint32_t* xdir, cudaStream_t stream);

// Self-test of the bounded device waits (see cga_selftest_wait_timeout).
size_t wait_selftest_bytes();
cudaError_t run_wait_selftest(void* scratch, cudaStream_t stream);

int device_sm_count();

// Launch accounting (cga_kernel_launches).
void count_launch(unsigned n);

}  // namespace libcga
