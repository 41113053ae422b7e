/*
 * libcga -- compressed geometric arrays (CGA) on one GB300 (sm_103a).
 *
 * C ABI of the hot path of "Compressed Geometric Arrays for Point Cloud
 * Processing" (Roodaki & Nazm Bojnordi): quantize float32 points to a voxel
 * grid, encode and sort them into the CGA layout of Sec. V, and run the CGA
 * operations of Sec. V-A..C (merge, orthogonal projection, exact nearest
 * neighbour) plus lossless decode.  Every step runs in hand-written CUDA
 * kernels; the host side only validates arguments, allocates and launches.
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are DEVICE pointers (current device); h_* are host.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is stream-ordered and asynchronous: a call returns once its kernels
 *    are queued.  Only cga_info / cga_view / cga2d_info / cga2d_view wait.
 *  - Handles (cga_t, cga2d_t) own their device arrays, obtained from the
 *    caller's allocator (NULL allocator = cudaMallocAsync/cudaFreeAsync on the
 *    call's stream).  Release them with cga_free / cga2d_free.
 *  - Errors: every call returns CGA_OK (0) or a negative CGA_ERR_* code and
 *    never aborts the process.  Argument errors are reported before any work
 *    is queued and leave *out untouched.  Errors found on the device while the
 *    queued work runs (non-finite input, a bounded wait that ran out) are
 *    recorded in the output handle and returned by the next cga_info /
 *    cga_view / cga2d_info on it; a merge or projection of a failed handle
 *    carries the error on to its output.
 *  - Coordinates: b = grid bits (1..16).  A voxel is (x, y, z), each in
 *    [0, 2^b); its key is x << 2b | y << b | z, and CGA order is ascending key
 *    order (x-major, then y, then z).  Coordinate arrays are uint16, pointer
 *    arrays uint32.
 */
#ifndef CGA_H
#define CGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CGA_OK 0
#define CGA_ERR_INVALID_ARG (-1)   /* bad size, bits, plane, grid, null pointer */
#define CGA_ERR_NONFINITE (-2)     /* NaN/Inf input point (or after transform) */
#define CGA_ERR_GRID_MISMATCH (-3) /* merge of CGAs on different grids */
#define CGA_ERR_OOM (-4)           /* the allocator returned NULL */
#define CGA_ERR_CUDA (-5)          /* a CUDA runtime call failed */
#define CGA_ERR_TIMEOUT (-6)       /* a bounded device wait ran out */
#define CGA_ERR_INTERNAL (-7)      /* a device-side consistency check failed */
#define CGA_ERR_CAPACITY (-8)      /* larger than a no-allocation call's fixed scratch */

/* Largest point count of one cloud (counts travel in 30-bit fields). */
#define CGA_MAX_POINTS ((uint64_t)((1u << 30) - 1u))

/* Voxel grid.  Quantization (the paper gives no formula; Sec. II-E-2-a asks
 * for a bounding box holding every point, Sec. VI-C uses QP = bits per axis):
 *   q_a = clamp(floorf(fmaf(p_a, scale, offset[a])), 0, 2^bits - 1)
 * evaluated in float32 with one rounding in the fma; the clamp keeps points on
 * or outside the box faces inside the grid. */
typedef struct {
  uint32_t bits;    /* 1..16 */
  float scale;      /* voxels per unit length, finite and > 0 */
  float offset[3];  /* finite */
} cga_grid;

/* Grid of a cube with lower corner lo[3] and edge `extent`:
 * scale = (float)2^bits / extent, offset[a] = -(lo[a] * scale).  Host only. */
int cga_grid_from_box(const float lo[3], float extent, uint32_t bits, cga_grid* out);

/* Device memory provider.  alloc returns a device pointer of at least `bytes`
 * bytes usable in stream order on `stream` (NULL on failure -> CGA_ERR_OOM,
 * nothing leaked); free releases one in stream order. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, void* stream);
} cga_allocator;

typedef struct cga cga_t;      /* a 3-level CGA (Sec. V) */
typedef struct cga2d cga2d_t;  /* a 2-level CGA of a projection (Sec. V-B) */

typedef struct {
  uint64_t h;         /* |X_index| distinct x                   */
  uint64_t g;         /* |Y_index| distinct (x, y) columns      */
  uint64_t u;         /* |Z_index| distinct voxels (points)     */
  uint64_t bytes;     /* 2h + 4(h+1) + 2g + 4(g+1) + 2u          */
  uint64_t capacity;  /* points the handle's buffers can hold   */
} cga_sizes;

typedef struct {
  cga_grid grid;
  uint64_t h, g, u;
  const uint16_t* X_index;    /* h     device */
  const uint32_t* X_pointer;  /* h + 1 device */
  const uint16_t* Y_index;    /* g     device */
  const uint32_t* Y_pointer;  /* g + 1 device */
  const uint16_t* Z_index;    /* u     device */
} cga_arrays;

typedef struct {
  uint32_t bits;
  int32_t plane;              /* CGA_PLANE_* */
  uint64_t h, g;              /* |U_index|, |V_index| */
  const uint16_t* U_index;    /* h     device */
  const uint32_t* U_pointer;  /* h + 1 device */
  const uint16_t* V_index;    /* g     device */
} cga2d_arrays;

#define CGA_PLANE_XY 0
#define CGA_PLANE_XZ 1
#define CGA_PLANE_YZ 2

/* Build (Sec. V, arrays; quantization as in cga_grid).
 * d_xyz: n points, float32 AoS (x, y, z), device, caller-owned, 4-byte
 *   aligned; n may be 0 (empty CGA: h = g = u = 0, X_pointer = Y_pointer = {0}).
 * h_xform12: NULL or 12 host floats, R (3x3 row-major) then t, applied first as
 *   p'_r = fmaf(R[r][0], x, fmaf(R[r][1], y, fmaf(R[r][2], z, t[r]))) -- the
 *   rigid transform that brings a view into the common frame before a merge
 *   (Sec. II-A).
 * *out: new handle; duplicate voxels are stored once.  Non-finite p or p'
 *   -> CGA_ERR_NONFINITE from the next cga_info.
 * Errors: INVALID_ARG (n > CGA_MAX_POINTS, bad grid, NULL out/d_xyz with n>0),
 *   OOM, CUDA. */
int cga_build(const float* d_xyz, uint64_t n, const cga_grid* g, const float* h_xform12,
              const cga_allocator* A, void* stream, cga_t** out);

/* Merge (Eq. 1, Sec. V-A): *out holds the set union of the voxels of a and
 * b, which must share one grid (bits, scale, offsets bit-identical), else
 * CGA_ERR_GRID_MISMATCH.  Either input may be empty. */
int cga_merge(const cga_t* a, const cga_t* b, const cga_allocator* A, void* stream,
              cga_t** out);

/* Orthogonal projection (Eq. 3 with m_x = m_y = 1, Sec. V-B) onto plane
 * CGA_PLANE_XY (keeps x, y), _XZ (x, z) or _YZ (y, z): *out holds the set of
 * distinct 2D voxels as a 2-level CGA, U_index/U_pointer over the first kept
 * axis and V_index over the second, ascending at both levels. */
int cga_project(const cga_t* a, int plane, const cga_allocator* A, void* stream,
                cga2d_t** out);

/* Exact nearest neighbour (Eq. 7-8, Sec. V-C).
 * d_q: m query points, float32 AoS, device.  Each query maps to the voxel
 *   floorf(fmaf(p_a, scale, offset_a)) of a's grid, clamped only to
 *   [-2^30, 2^30] (queries outside the box are allowed).
 * d_idx[j]: index, in CGA point order (the Z_index position), of the stored
 *   voxel with the least squared integer distance to query j; among equal
 *   distances the smaller key wins.  d_dist2[j]: that squared distance.
 *   Empty CGA or non-finite query: UINT32_MAX / UINT64_MAX.
 * Both output arrays hold m entries, device, caller-owned. */
int cga_nn_query(const cga_t* a, const float* d_q, uint64_t m, uint32_t* d_idx,
                 uint64_t* d_dist2, void* stream);

#define CGA_NN_MAX_LEVELS 2           /* coarse levels cga_nn_prepare_levels takes */
#define CGA_NN_MAX_SHIFT 12           /* largest coarse cell: 2^12 voxels per axis */
#define CGA_NN_AUTOTUNE_CANDIDATES 10 /* strategies cga_nn_autotune measures */
#define CGA_NN_TREE 0xFFFFFFFFu       /* shifts = {CGA_NN_TREE}, count 1: occupancy tree */

/* Build (once per CGA) the coarse levels that let NN search skip empty space.
 * Level k is the CGA of the occupied cells of 2^shifts[k] voxels per axis
 * (built by re-keying the next finer level), with, for each of its x slabs,
 * the index of the first slab of the next finer level inside it.  Afterwards
 * every NN call on `a` walks the coarsest level's cells outward from the query
 * and refines, level by level down to the CGA's own columns, only the cells
 * whose box lower bound can beat the best distance found so far (the results
 * do not change: the exact nearest voxel, ties to the smaller key).
 * Every call also builds (once) an x directory per level: for each x value v
 * the index of the first X_index entry >= v -- the dense per-x table of
 * G-Arrays (Sec. V) used only to start a slab walk in one lookup
 * (4 * (2^bits + 1) bytes for the CGA itself), and a column table of the
 * CGA: per column its voxel range and its lowest and highest z, 16 bytes per
 * column of capacity, read by one load when a search visits the column.
 * shifts: count (0..CGA_NN_MAX_LEVELS) strictly increasing values in
 * 1..min(CGA_NN_MAX_SHIFT, bits-1), host memory; count 0 drops the coarse
 * levels and keeps only the x directory (fine search).
 * shifts = {CGA_NN_TREE} with count 1 builds, instead of coarse levels, an
 * occupancy tree: a 64-ary tree in which a node of level l is a cell of 4^l
 * voxels per axis that records which of its 4 x 4 x 4 sub-cells hold a voxel
 * (a level-1 node, a brick, records its 64 voxels), ceil(bits / 2) levels.
 * NN calls then descend it nearest child first and skip every cell whose box
 * lies farther than the best voxel found so far (same exact results; for
 * queries far from every voxel, e.g. a surface in a large box, this visits
 * far fewer cells than the slab walk).  It is built on the device by a sort
 * of the voxels' tree keys and one compaction per level; its arrays take 8
 * bytes per brick and 16 per node of each higher level, reserved by the
 * capacity bounds (at most the CGA's capacity or the level's cell count per
 * level).
 * Replaces any earlier preparation.  Memory comes from a's allocator and is
 * released with a.  Stream-ordered.  CGA_ERR_INVALID_ARG for a view handle or
 * bad shifts. */
int cga_nn_prepare_levels(cga_t* a, const uint32_t* shifts, uint32_t count, void* stream);

/* cga_nn_prepare_levels with one coarse level of 2^shift voxel cells, or none
 * when shift is 0. */
int cga_nn_prepare(cga_t* a, uint32_t shift, void* stream);

/* Pick the NN search strategy for `a` by measurement: run the m sample queries
 * d_q (device; a few tens of thousands representative queries suffice) under
 * each candidate and keep the fastest prepared on `a`.  Candidates, in order
 * (coarse shifts): none (fine search alone); 2; 3; 4; 5; 2,5; 3,6; 3,7; 4,8;
 * CGA_NN_TREE (the occupancy tree).
 * chosen_shifts (CGA_NN_MAX_LEVELS entries) receives the winner's shifts, 0
 * for an unused level ({CGA_NN_TREE, 0} for the tree).  times_ms (NULL or CGA_NN_AUTOTUNE_CANDIDATES floats)
 * receives each candidate's time, -1 for one the grid cannot take.  Waits for
 * the timings. */
int cga_nn_autotune(cga_t* a, const float* d_q, uint64_t m, uint32_t* chosen_shifts,
                    float* times_ms, void* stream);

/* cga_nn_autotune for a CGA that is prepared once per m_per_prepare queries
 * (for instance rebuilt every step and searched by that many): a candidate's
 * cost is its preparation time plus the sample's search time scaled by
 * m_per_prepare / m, and times_ms receives that cost.  m_per_prepare == 0 is
 * cga_nn_autotune (the search alone). */
int cga_nn_autotune_for(cga_t* a, const float* d_q, uint64_t m, uint64_t m_per_prepare,
                        uint32_t* chosen_shifts, float* times_ms, void* stream);

/* The two halves of cga_nn_query, for callers that reuse one query order or
 * time the search on its own.  cga_nn_sort_queries writes m 64-bit keys
 * (30-bit Morton code of the query's grid voxel << 32 | query index), sorted
 * ascending, to d_order (device, m entries; scratch from a's allocator).
 * cga_nn_query_ordered answers the queries in the order d_order gives (low 32
 * bits = query index; NULL = index order); results land at each query's own
 * index and equal cga_nn_query's.  Indices >= m in d_order are skipped. */
int cga_nn_sort_queries(const cga_t* a, const float* d_q, uint64_t m, uint64_t* d_order,
                        void* stream);
int cga_nn_query_ordered(const cga_t* a, const float* d_q, uint64_t m, const uint64_t* d_order,
                         uint32_t* d_idx, uint64_t* d_dist2, void* stream);

/* cga_nn_query without any memory allocation.  (The paper has no counterpart:
 * this is a deployment variant of the NN call above, same results bit for
 * bit.)  For callers that cannot allocate device memory when they query --
 * under a memory budget reserved in advance, inside real-time loops where
 * cudaMalloc's device-wide synchronization and unbounded latency are not
 * allowed, or where another framework owns the allocator.
 * The scratch of the query sort comes from one fixed __device__ array of
 * 18 MiB built into the library; every GPU that loads the library holds it
 * until the process exits.  m must be <= CGA_NOALLOC_MAX_QUERIES, else
 * CGA_ERR_CAPACITY and nothing is queued.  The caller passes the CGA, the
 * queries and the outputs exactly as for cga_nn_query.
 * The first call on a device looks up the array's device address (once per
 * device).  Each call copies its small segment tables from host memory into
 * the array (cudaMemcpyAsync).  A search structure that cga_nn_prepare_levels
 * built on `a` (x directory, column table, coarse levels or occupancy tree)
 * is used as cga_nn_query uses it.  All calls share
 * the one array and each call resets what it needs, so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race:
 * serialize them, e.g. on one stream.  Nothing is allocated: no cudaMalloc,
 * cudaFree, pool or allocator callback. */
#define CGA_NOALLOC_MAX_QUERIES ((uint64_t)1 << 20)
int cga_nn_query_noalloc(const cga_t* a, const float* d_q, uint64_t m, uint32_t* d_idx,
                         uint64_t* d_dist2, void* stream);

/* Decode (lossless inverse of the build, CGA order): d_xyz receives u triples
 * (x, y, z) as uint32, u from cga_info; device, caller-owned, >= 3u entries
 * (may be NULL when the handle's capacity is 0). */
int cga_decode(const cga_t* a, uint32_t* d_xyz, void* stream);

/* ---- Value (attribute) array, Sec. V --------------------------------------
 * A CGA may carry one row of `channels` (1..CGA_MAX_CHANNELS) uint8
 * attributes per stored voxel, in CGA point order: row p belongs to
 * Z_index[p].  Several points quantized into one voxel give it the
 * round-half-up integer mean (sum + k/2) / k of their k rows per channel
 * (Sec. III-B: the colours of the points merged into one box are averaged), or the
 * row of the first of them in input order.  A merge keeps, for a voxel held by
 * both inputs, the base's (a's) row or (a + b + 1) / 2 per channel (Sec. II-A);
 * a voxel held by one input keeps its row. */
#define CGA_MAX_CHANNELS 4
#define CGA_VALUE_AVERAGE 0
#define CGA_VALUE_FIRST 1
#define CGA_MERGE_BASE 0
#define CGA_MERGE_AVERAGE 1

/* cga_build plus the Value array.  d_attr: n * channels uint8 rows, device,
 * point order (the same points as d_xyz).  Each point finds its voxel by the
 * Sec. V-A lookup; sums are exact integers, so the result does not depend
 * on arrival order.  Errors as cga_build; CGA_ERR_INVALID_ARG for channels or
 * policy out of range or a NULL d_attr with n > 0. */
int cga_build_values(const float* d_xyz, const uint8_t* d_attr, uint32_t channels, uint64_t n,
                     const cga_grid* g, const float* h_xform12, int policy,
                     const cga_allocator* A, void* stream, cga_t** out);

/* cga_merge plus the Value array (a is the base).  Both inputs must carry
 * values with the same channel count (else CGA_ERR_INVALID_ARG). */
int cga_merge_values(const cga_t* a, const cga_t* b, int policy, const cga_allocator* A,
                     void* stream, cga_t** out);

/* Device pointer to a's Value array (u * channels bytes, valid while a
 * lives; stream-ordered after the call that made a) and its channel count;
 * NULL and 0 when a has no values. */
int cga_values(const cga_t* a, const uint8_t** d_values, uint32_t* channels);

/* ---- Radius search (the Eq. 8 set within a radius) -------------------------
 * Query voxels as for cga_nn_query.  Query j's result is every stored voxel
 * with squared integer distance <= r2 (voxel units), in ascending CGA index.
 * cga_radius_count writes d_offsets (m + 1 uint64, device): the exclusive
 * prefix of the per-query counts, d_offsets[m] = the total (read it to size
 * the outputs).  cga_radius_fill then writes query j's voxels at
 * [d_offsets[j], d_offsets[j + 1]) of d_idx (CGA index) and d_dist2.  A
 * non-finite query has none.  r2 <= CGA_MAX_RADIUS2. */
#define CGA_MAX_RADIUS2 (1ull << 62)
int cga_radius_count(const cga_t* a, const float* d_q, uint64_t m, uint64_t r2,
                     uint64_t* d_offsets, void* stream);
int cga_radius_fill(const cga_t* a, const float* d_q, uint64_t m, uint64_t r2,
                    const uint64_t* d_offsets, uint32_t* d_idx, uint64_t* d_dist2,
                    void* stream);

/* k nearest stored voxels of each query: the k least (squared integer
 * distance, key) pairs, ascending, at d_idx / d_dist2 [j * k, j * k + k)
 * (device, m * k entries each).  Slots past the number of stored voxels,
 * and all slots of a non-finite query, hold UINT32_MAX / UINT64_MAX.
 * k = 1 is cga_nn_query's answer.  1 <= k <= CGA_KNN_MAX_K (the paper's
 * Fig. 3 shows 400 neighbours). */
#define CGA_KNN_MAX_K 1024
int cga_knn(const cga_t* a, const float* d_q, uint64_t m, uint32_t k, uint32_t* d_idx,
            uint64_t* d_dist2, void* stream);

/* ---- Compression pieces (Sec. V-D) and the G-Arrays X pointer (Sec. V) -------
 * Sec. V-D predicts a frame from a reference frame: both are clustered,
 * each cluster's centroid motion is a motion vector, the predicted frame's
 * points are moved by their cluster's vector, and each moved point is matched
 * to its corresponding point of the reference by a search of the reference's
 * CGA.  Here the clustering runs on a CGA's stored voxels (integers), with
 * results independent of the visiting order:
 *
 * cga_kmeans: k-means (Lloyd passes) with the eight centres first placed at
 * the corners of the voxels' bounding box (corner c: the greatest coordinate
 * of axis a where bit a of c is set, else the least).  Centres are int64 in
 * 1/256 voxel; a pass labels every voxel with the centre of least squared
 * distance (ties: the lower cluster) and stops the run if it changed no label
 * (after the first pass); otherwise each non-empty cluster's centre becomes
 * (256 * sum + n / 2) / n per axis (empty clusters keep theirs).  At most
 * max_iter (1..CGA_KMEANS_MAX_ITER) passes.  Outputs (device): d_label[u]
 * (0..7, CGA order), d_centres[8 * 3], d_counts[8] (voxels per cluster in the
 * last pass), *d_iters (passes done; 0 for an empty CGA, whose centres and
 * counts are 0).  Stream-ordered, no host synchronization.
 *
 * cga_motion_vectors: d_mv[c * 3 + a] = ref - pred centre (1/256 voxel) for
 * every cluster non-empty in both frames, else 0 (8 * 3 int64, device).
 *
 * cga_reconstruct: the predicted frame moved by its clusters' vectors:
 * d_out[3 i + a] = voxel_a(i) + floor((mv[label(i)][a] + 128) / 256), int32,
 * u * 3 (not clamped to the grid).  Labels must be 0..7.
 *
 * cga_nn_query_voxels: cga_nn_query for integer query voxels (d_qv: m * 3
 * int32, each clamped to +-2^30), e.g. the reconstructed frame against the
 * reference's CGA: the corresponding point of each reconstructed voxel.
 *
 * cga_lookup: the Sec. V-A point lookup of integer voxels: d_idx[j] = CGA
 * index of voxel j, or UINT32_MAX when it is not stored (or off the grid).
 *
 * cga_garrays_x: the X pointer in the G-Arrays form (one cell per x value
 * of the whole axis, which Sec. V contrasts with the CGA's compact X_index +
 * X_pointer): d_xptr[v] = number of (x, y) columns with x < v, for v in
 * [0, 2^bits] (2^bits + 1 uint32, device).  cga_garrays_lookup answers
 * cga_lookup through it (x indexes the pointer array directly).
 *
 * cga_residual: the residual frame of Sec. V-D: for each point i of the
 * reconstructed frame (u_pred points, values d_pred_values, channels per
 * point) and its corresponding reference point d_idx[i] (e.g. from
 * cga_nn_query_voxels; the reference has u_ref points, values d_ref_values):
 * d_out[i * channels + c] = pred - ref (int16), or pred itself when d_idx[i]
 * >= u_ref (no corresponding point).  All device pointers; channels 1..4. */
#define CGA_KMEANS_MAX_ITER 1024
int cga_kmeans(const cga_t* a, uint32_t max_iter, uint8_t* d_label, int64_t* d_centres,
               uint64_t* d_counts, uint32_t* d_iters, void* stream);
int cga_motion_vectors(const int64_t* d_ref_centres, const uint64_t* d_ref_counts,
                       const int64_t* d_pred_centres, const uint64_t* d_pred_counts,
                       int64_t* d_mv, void* stream);
int cga_reconstruct(const cga_t* pred, const uint8_t* d_label, const int64_t* d_mv,
                    int32_t* d_out, void* stream);
int cga_nn_query_voxels(const cga_t* a, const int32_t* d_qv, uint64_t m, uint32_t* d_idx,
                        uint64_t* d_dist2, void* stream);
int cga_lookup(const cga_t* a, const int32_t* d_qv, uint64_t m, uint32_t* d_idx, void* stream);
int cga_residual(const uint8_t* d_pred_values, uint64_t u_pred, const uint8_t* d_ref_values,
                 uint64_t u_ref, const uint32_t* d_idx, uint32_t channels, int16_t* d_out,
                 void* stream);
int cga_garrays_x(const cga_t* a, uint32_t* d_xptr, void* stream);
int cga_garrays_lookup(const cga_t* a, const uint32_t* d_xptr, const int32_t* d_qv, uint64_t m,
                       uint32_t* d_idx, void* stream);

/* ---- Perspective projection (Eq. 5-6) ---------------------------------------
 * Each stored voxel (x, y, z) is taken to the eye's frame, s = (x - eye[0],
 * y - eye[1], z - eye[2]) (float, voxel units), rotated about the y axis by
 * the angle whose cosine and sine are cos_t, sin_t (Eq. 6: x' = cos*sx -
 * sin*sz, z' = sin*sx + cos*sz, y' = sy) and divided onto the plane at
 * distance D (Eq. 5: px = D*x'/z', py = D*y'/z').  Voxels with z' <= 0 are
 * dropped.  Pixel (floor(px + W/2), floor(py + H/2)) of the W x H image keeps
 * the voxel of least z', ties to the smaller CGA index.  Each step is one IEEE
 * float operation in this order: fmaf(cos, sx, (-sin)*sz), fmaf(sin, sx,
 * cos*sz), (D*x')/z', floor(px + W/2).
 * d_index (W*H, device): CGA index of the pixel's voxel or UINT32_MAX;
 * d_depth (W*H, device): its z' or +inf.  Row-major (v*W + u).  Scratch of
 * 8*W*H bytes from a's allocator. */
#define CGA_MAX_PIXELS (1ull << 28)
int cga_perspective(const cga_t* a, const float eye[3], float cos_t, float sin_t, float D,
                    uint32_t W, uint32_t H, uint32_t* d_index, float* d_depth, void* stream);

/* ---- Batched forms: one set of kernel launches serves every item. --------
 * Each item has the semantics of the single call; handles are independent
 * (free each one).  On an error nothing is returned and no handle leaks. */

typedef struct {
  const float* d_xyz;      /* n points, device */
  uint64_t n;
  cga_grid grid;
  const float* h_xform12;  /* NULL or 12 host floats, as in cga_build */
} cga_cloud;

/* cga_build for `count` clouds (grids may differ) -> out[count]. */
int cga_build_batch(const cga_cloud* clouds, uint32_t count, const cga_allocator* A,
                    void* stream, cga_t** out);

/* cga_merge of a[i] and b[i] for every i -> out[count]. */
int cga_merge_batch(const cga_t* const* a, const cga_t* const* b, uint32_t count,
                    const cga_allocator* A, void* stream, cga_t** out);

/* cga_project of a[i] onto planes[i] for every i -> out[count]. */
int cga_project_batch(const cga_t* const* a, const int* planes, uint32_t count,
                      const cga_allocator* A, void* stream, cga2d_t** out);

typedef struct {
  const float* d_q;   /* m query points, device */
  uint64_t m;
  uint32_t* d_idx;    /* m, device */
  uint64_t* d_dist2;  /* m, device */
} cga_queries;

/* cga_nn_query of q[i] against a[i] for every i (scratch from A). */
int cga_nn_query_batch(const cga_t* const* a, const cga_queries* q, uint32_t count,
                       const cga_allocator* A, void* stream);

/* ---- Launch-shape tuning ---------------------------------------------------
 * The sort (build, xz/yz projection, NN coarse levels) and merge kernels run
 * in one of several launch shapes, all with identical results.  A
 * process-wide table keyed by (grid bits, bit length of the element count)
 * holds the shape each call uses: the sort looks up (bits, n) of its largest
 * input, the merge (bits, capacity of A + capacity of B); a batch looks up
 * its largest item; a pipeline looks up (largest bits, largest n) once at
 * create, for its sort and its merge alike.
 * Entries default to {8, 512, 2048}.  Host-only and thread-safe. */
typedef struct {
  uint32_t radix_bits;    /* digit width of an LSD pass: 8 or 9 (9 needs sort_threads 512) */
  uint32_t sort_threads;  /* threads per 4096-key tile: 256 (16 keys each) or 512 (8 keys each) */
  uint32_t merge_half;    /* merge-path partition: a splitter every 512, 1024 or 2048 points
                             of each input (tiles of at most 2 * merge_half keys) */
} cga_tuning;

#define CGA_TUNE_SORT_CANDIDATES 3  /* (8, 256), (8, 512), (9, 512) */
#define CGA_TUNE_MERGE_CANDIDATES 3 /* 512, 1024, 2048 */

/* Set (t != NULL) or clear (t == NULL: back to the default) the entry for
 * grids of `bits` per axis and element counts with n's bit length.
 * CGA_ERR_INVALID_ARG for bits outside 1..16 or a shape not listed above. */
int cga_tuning_set(uint32_t bits, uint64_t n, const cga_tuning* t);
/* The shape a call with (bits, n) would use now. */
int cga_tuning_get(uint32_t bits, uint64_t n, cga_tuning* out);

/* Fill the entry for (g->bits, n) by measurement on the caller's cloud d_xyz
 * (n >= 2 float32 points, device): time a build of the whole cloud under each
 * sort candidate, then the merge of the CGAs of its two halves under each
 * merge candidate, and keep the fastest of each.  chosen receives the stored
 * shape; times_ms (NULL or CGA_TUNE_SORT_CANDIDATES + CGA_TUNE_MERGE_CANDIDATES
 * floats) each candidate's least time of two runs, in the order listed above.
 * Allocates from the library pool, waits for the timings; on an error the
 * entry is left as it was. */
int cga_autotune(const float* d_xyz, uint64_t n, const cga_grid* g, cga_tuning* chosen,
                 float* times_ms, void* stream);

/* ---- Pre-planned pipeline (capturable) ------------------------------------
 * For each item i: build the cloud, build its twin (the same points under the
 * rigid transform xform12, the view brought into the common frame of
 * Sec. II-A), merge the two (Eq. 1), project the merge onto the xy plane
 * (Eq. 3) and answer m NN queries against the merge (Eq. 7-8).  Create does
 * every allocation (one arena from A) and uploads every descriptor; run then
 * only queues memsets and kernels -- about twenty launches for all items, each
 * launch covering every cloud -- so it is safe to capture in a CUDA graph.
 * The inputs (points, queries) are read and the NN outputs written at the
 * device addresses given at create, on every run. */
typedef struct cga_pipeline cga_pipeline_t;

typedef struct {
  const float* d_xyz;  /* n points, device */
  uint64_t n;          /* <= CGA_MAX_POINTS / 2 */
  cga_grid grid;
  float xform12[12];   /* twin transform: R row-major, then t */
  const float* d_q;    /* m NN queries, device (may be NULL when m == 0) */
  uint64_t m;
  uint32_t* d_idx;     /* m, device */
  uint64_t* d_dist2;   /* m, device */
} cga_pipeline_item;

/* cga_autotune for a pipeline: create the pipeline of these items under each
 * sort candidate, then each merge candidate, time two graph replays of each
 * (after the capturing one) and store the fastest shape in the entry the
 * pipeline looks up, (largest bits, largest n).  chosen and times_ms as in
 * cga_autotune.  Every candidate pipeline is freed before the next is made;
 * the items' NN outputs are overwritten. */
int cga_pipeline_autotune(const cga_pipeline_item* items, uint32_t count, cga_tuning* chosen,
                          float* times_ms, void* stream);

/* Plan `count` items; waits until the descriptors are on the device. */
int cga_pipeline_create(const cga_pipeline_item* items, uint32_t count, const cga_allocator* A,
                        void* stream, cga_pipeline_t** out);
/* Queue one pass of every stage on `stream`. */
int cga_pipeline_run(cga_pipeline_t* p, void* stream);
/* First call captures cga_pipeline_run into a CUDA graph (on a private
 * stream); every call launches that graph on `stream`. */
int cga_pipeline_run_graph(cga_pipeline_t* p, void* stream);
/* Non-owning handles of item i's results (which: 0 cloud, 1 twin, 2 merged),
 * valid until cga_pipeline_free; they refresh on every run.  cga_free on them
 * does nothing. */
int cga_pipeline_view(const cga_pipeline_t* p, uint32_t i, int which, const cga_t** out);
int cga_pipeline_view_xy(const cga_pipeline_t* p, uint32_t i, const cga2d_t** out);
void cga_pipeline_free(cga_pipeline_t* p);

/* ---- Served loop: continuous batching over device-resident CGAs ----------
 * A scheduler thread keeps `slots` CUDA streams busy.  Whenever a stream is
 * idle and requests are pending, it batches requests from the head of the
 * queue (arrival order) while their device-memory footprint fits what is left
 * of `memory_budget`, up to `max_batch` per batch.  All NN requests of a batch
 * share one segmented NN launch set; all merge+project requests one batched
 * merge (Eq. 1) and one batched projection (Eq. 3).  Requests that arrive while
 * batches run are admitted onto free streams as memory frees up, so their work
 * overlaps on the GPU.  Results equal the plain single calls bit for bit. */
typedef struct cga_server cga_server_t;

#define CGA_REQ_NN 0             /* m NN queries against pool[a] */
#define CGA_REQ_MERGE_PROJECT 1  /* merge pool[a] with pool[b], project onto plane */

typedef struct {
  int32_t kind;
  uint32_t a, b;       /* pool indices (b: merge+project only) */
  int32_t plane;       /* merge+project: CGA_PLANE_* */
  const float* d_q;    /* NN: m queries, device; must stay valid until done */
  uint64_t m;
  uint32_t* d_idx;     /* NN outputs, device, m entries */
  uint64_t* d_dist2;
} cga_request;

typedef struct {
  uint64_t ticket;       /* from cga_server_submit */
  int32_t status;        /* CGA_OK or an error code */
  uint64_t t_submit_ns;  /* cga_now_ns() clock: arrival */
  uint64_t t_start_ns;   /* batch queued on a stream */
  uint64_t t_done_ns;    /* completion seen by the scheduler */
  cga_t* merged;         /* merge+project results: the caller frees them */
  cga2d_t* projected;
} cga_completion;

typedef struct {
  uint64_t memory_budget;  /* bytes of scratch + outputs in flight at once */
  uint32_t slots;          /* concurrent batches (CUDA streams), 1..64 */
  uint32_t max_batch;      /* requests per batch */
} cga_server_config;

/* pool: CGAs that stay resident and unchanged while the server lives (the
 * call waits until they are built).  Scratch and results come from A. */
int cga_server_create(const cga_t* const* pool, uint32_t count, const cga_server_config* cfg,
                      const cga_allocator* A, cga_server_t** out);
/* Thread-safe, non-blocking.  A request larger than the whole budget is
 * refused with CGA_ERR_OOM; merge of pool CGAs on different grids with
 * CGA_ERR_GRID_MISMATCH. */
int cga_server_submit(cga_server_t* s, const cga_request* r, uint64_t* ticket);
/* Up to `max` finished requests (oldest first); non-blocking. */
int cga_server_poll(cga_server_t* s, cga_completion* out, uint32_t max, uint32_t* n);
/* Wait until every submitted request has finished. */
int cga_server_drain(cga_server_t* s);
/* Finish outstanding work, free unpolled results, stop the scheduler. */
void cga_server_free(cga_server_t* s);
/* The server's clock (steady, nanoseconds). */
uint64_t cga_now_ns(void);

/* Sizes of a handle; waits for the work that produced it.  Returns the
 * device-side error recorded for the handle, if any. */
int cga_info(const cga_t* a, cga_sizes* out);

/* Device pointers of the geometry arrays (valid until cga_free); waits like
 * cga_info. */
int cga_view(const cga_t* a, cga_arrays* out);

int cga2d_info(const cga2d_t* p, uint64_t* h, uint64_t* g);
int cga2d_view(const cga2d_t* p, cga2d_arrays* out);

/* Copy the geometry arrays to caller-owned HOST buffers sized from cga_info
 * (X_index h, X_pointer h+1, Y_index g, Y_pointer g+1, Z_index u entries);
 * waits like cga_info.  A CGA is its own serialized form: these five arrays
 * and the grid rebuild it exactly. */
int cga_download(const cga_t* a, uint16_t* h_X_index, uint32_t* h_X_pointer,
                 uint16_t* h_Y_index, uint32_t* h_Y_pointer, uint16_t* h_Z_index);
int cga2d_download(const cga2d_t* p, uint16_t* h_U_index, uint32_t* h_U_pointer,
                   uint16_t* h_V_index);

/* Release a handle in stream order on the stream of the call that made it. */
void cga_free(cga_t* a);
void cga2d_free(cga2d_t* p);

/* Self-test of the bounded device waits: queues one radix-sort tile whose
 * predecessor tile never runs, so the look-back word it waits on is never
 * published.  The wait gives up after its limit (about one second), records
 * the timeout and the kernel returns; *observed receives the status the tile
 * recorded (CGA_ERR_TIMEOUT when the bound works) and the device stays usable.
 * Waits for the result. */
int cga_selftest_wait_timeout(void* stream, int* observed);

/* Number of kernels this library has queued since the process started (all
 * devices, all threads); a cheap counter for launch accounting. */
uint64_t cga_kernel_launches(void);

/* Static description of an error code. */
const char* cga_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
