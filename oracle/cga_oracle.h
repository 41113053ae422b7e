/*
 * CPU oracle for the compressed-geometric-array (CGA) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, slow, single-threaded C++17 code is
 * the reference the CUDA library is checked against.  It shares no code,
 * header, table or helper with the CUDA path, and only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  The product path
 * never calls it and has no CPU fallback.
 *
 * Every function states the passage of the paper it follows ("Compressed
 * Geometric Arrays for Point Cloud Processing", Roodaki & Nazm Bojnordi):
 *   Sec. V (CGA arrays and their recurrences), Sec. V-A (point lookup and
 *   merge), Sec. V-B (projection), Sec. V-C (NN search), Eq. 1 (merge as a
 *   set union), Eq. 3 (orthogonal projection), Eq. 7-8 (Euclidean distance and
 *   the NN set), Sec. II-E-2-a (bounding box including all points), Sec. V-D
 *   (clustering with corner-seeded k-means, cluster motion vectors and the
 *   reconstructed frame matched to the reference by NN), and the G-Arrays
 *   form of X_pointer that Sec. V contrasts with the CGA.
 *
 * Parity pinned: every function here is pinned by the not-gpu tests against
 * hand-written fixtures, closed forms, invariants and independent library
 * routines (numpy set/sort routines, exhaustive search).
 */
#ifndef CGA_ORACLE_H
#define CGA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG (-1)
#define ORC_ERR_NONFINITE (-2)

/* A CGA as six-array storage minus the attribute (Value) array: caller-owned
 * host buffers.  Sizes: h = |X_index|, g = |Y_index|, u = |Z_index|;
 * X_pointer has h+1 entries and Y_pointer g+1 entries. */
typedef struct {
  uint32_t bits;
  uint64_t h, g, u;
  uint16_t* X_index;
  uint32_t* X_pointer;
  uint16_t* Y_index;
  uint32_t* Y_pointer;
  uint16_t* Z_index;
} orc_cga;

/* 2-level CGA of a projection onto a coordinate plane: U_index (distinct
 * first kept coordinate), U_pointer (h2+1), V_index (g2). */
typedef struct {
  uint32_t bits;
  uint64_t h, g;
  uint16_t* U_index;
  uint32_t* U_pointer;
  uint16_t* V_index;
} orc_cga2d;

/* Grid from a cubic box with lower corner lo[] and edge length extent:
 * scale = 2^bits / extent, offset[a] = -(lo[a] * scale), all in float. */
int orc_grid_from_box(const float lo[3], float extent, uint32_t bits,
                      float* scale, float offset[3]);

/* Quantize + encode: keys[i] = x << 2b | y << b | z.  xform12 (nullable) is
 * R (3x3 row-major) followed by t (3). */
int orc_quantize(const float* xyz, uint64_t n, uint32_t bits, float scale,
                 const float offset[3], const float* xform12, uint64_t* keys);

/* CGA arrays from a sorted, duplicate-free key list (Sec. V recurrences).
 * Output buffers must hold u entries (X_pointer/Y_pointer u+1). */
int orc_from_sorted_keys(const uint64_t* keys, uint64_t u, uint32_t bits,
                         orc_cga* out);

/* Build: quantize, sort, drop duplicates, arrays.  Buffers hold n (n+1). */
int orc_build(const float* xyz, uint64_t n, uint32_t bits, float scale,
              const float offset[3], const float* xform12, orc_cga* out);

/* Decode to (x, y, z) uint32 triples in CGA order (u * 3 entries). */
int orc_decode(const orc_cga* a, uint32_t* xyz);

/* Decode to keys in CGA order (u entries). */
int orc_decode_keys(const orc_cga* a, uint64_t* keys);

/* Point lookup (Sec. V-A): index in CGA point order, or -1. */
int64_t orc_lookup(const orc_cga* a, uint32_t x, uint32_t y, uint32_t z);

/* Merge (Eq. 1, Sec. V-A).  out buffers hold a->u + b->u (+1). */
int orc_merge(const orc_cga* a, const orc_cga* b, orc_cga* out);

/* Orthogonal projection (Eq. 3 with m = 1, Sec. V-B) onto plane
 * 0 = xy, 1 = xz, 2 = yz.  out buffers hold a->u (+1). */
int orc_project(const orc_cga* a, int plane, orc_cga2d* out);

/* Exact NN (Eq. 7-8) by exhaustive search over every stored voxel.
 * Query voxel: floorf(fmaf(p, scale, offset)) clamped to [-2^30, 2^30].
 * idx = CGA point index of the nearest voxel (ties: smaller key), dist2 =
 * squared integer distance.  Empty CGA or non-finite query: idx = UINT32_MAX,
 * dist2 = UINT64_MAX. */
int orc_nn_brute(const orc_cga* a, float scale, const float offset[3],
                 const float* q, uint64_t m, uint32_t* idx, uint64_t* dist2);

/* Query voxels of m points (the NN reading above): out[3j+a] =
 * floorf(fmaf(q, scale, offset_a)) clamped to [-2^30, 2^30]; valid[j] = 0 for a
 * non-finite query (its out entries are 0). */
int orc_query_voxels(const float* q, uint64_t m, float scale, const float offset[3],
                     int64_t* out, uint8_t* valid);

/* Exact NN by the CGA procedure of Sec. V-C: exact-match lookup, else the
 * nearest x -> nearest y -> nearest z bound, then every voxel inside the
 * per-axis window of that bound.  Same outputs as orc_nn_brute. */
int orc_nn_window(const orc_cga* a, float scale, const float offset[3],
                  const float* q, uint64_t m, uint32_t* idx, uint64_t* dist2);

/* ---- Value (attribute) array, Sec. V ------------------------------------
 * Every stored voxel carries `channels` (1..4) uint8 attributes, in CGA point
 * order (values[p * channels + c] belongs to Z_index[p]). */
#define ORC_VALUE_AVERAGE 0 /* Sec. III-B (pcdownsample): the points of one voxel are averaged */
#define ORC_VALUE_FIRST 1   /* the voxel keeps the attributes of its first input point */
#define ORC_MERGE_BASE 0    /* Sec. II-A: an overlapping voxel keeps the base cloud's (a's) */
#define ORC_MERGE_AVERAGE 1 /* Sec. II-A: or the average of the two */

/* Build with values.  attr: n * channels input attributes in point order.
 * The average of a voxel's k points is the round-half-up integer mean
 * (sum + k / 2) / k per channel; FIRST keeps the lowest input index.
 * values: n * channels entries (u * channels are written). */
int orc_build_values(const float* xyz, const uint8_t* attr, uint32_t channels, uint64_t n,
                     uint32_t bits, float scale, const float offset[3], const float* xform12,
                     int policy, orc_cga* out, uint8_t* values);

/* Merge with values (Eq. 1 with the Sec. II-A attribute rule; a is the base).
 * The average of a voxel present in both is (va + vb + 1) / 2 per channel.
 * out and values hold a->u + b->u entries (values times channels). */
int orc_merge_values(const orc_cga* a, const uint8_t* va, const orc_cga* b, const uint8_t* vb,
                     uint32_t channels, int policy, orc_cga* out, uint8_t* values);

/* ---- Perspective projection (Eq. 5-6, rotation about y) --------------------
 * Each stored voxel (x, y, z) becomes s = (x - ex, y - ey, z - ez) in float
 * (voxel units, eye e), is rotated about the y axis by theta (Eq. 6 matrix:
 * x' = cos*sx - sin*sz, z' = sin*sx + cos*sz, y' = sy; cos and sin given as
 * floats) and projected onto the plane at distance D (Eq. 5): px = D*x'/z',
 * py = D*y'/z'.  Voxels with z' <= 0 are behind the eye and dropped.  Pixel
 * (floor(px + W/2), floor(py + H/2)) inside a W x H image keeps the voxel of
 * least z' (ties: the smaller CGA index).  Every step is one float
 * operation in this order: fmaf(cos, sx, (-sin)*sz) and fmaf(sin, sx, cos*sz)
 * for the rotation, (D*x')/z' for the projection, floor(px + W/2) for the
 * pixel.  Outputs: index[v*W+u] = CGA index or UINT32_MAX, depth[v*W+u] = z'
 * (+inf when empty). */
int orc_perspective(const orc_cga* a, const float eye[3], float cos_t, float sin_t, float D,
                    uint32_t W, uint32_t H, uint32_t* index, float* depth);

/* ---- Radius search and k-NN (the Eq. 8 set generalised) --------------------
 * Query voxels as for NN.  Radius: every stored voxel with squared integer
 * distance <= r2, in ascending CGA index.  counts[j] = how many; fill writes
 * query j's voxels at [offsets[j], offsets[j] + counts[j]).  Non-finite query:
 * none.  k-NN: the k stored voxels of least (distance^2, key), ascending; slots
 * beyond the number of stored voxels (or for a non-finite query) hold
 * UINT32_MAX / UINT64_MAX.  idx and dist2 hold m * k entries. */
int orc_radius_count(const orc_cga* a, float scale, const float offset[3], const float* q,
                     uint64_t m, uint64_t r2, uint64_t* counts);
int orc_radius_fill(const orc_cga* a, float scale, const float offset[3], const float* q,
                    uint64_t m, uint64_t r2, const uint64_t* offsets, uint32_t* idx,
                    uint64_t* dist2);
int orc_knn(const orc_cga* a, float scale, const float offset[3], const float* q, uint64_t m,
            uint32_t k, uint32_t* idx, uint64_t* dist2);

/* ---- Compression pieces (Sec. V-D) and the G-Arrays form (Sec. V) -------
 * Integer query voxels qv (m * 3 int32, any value).
 * lookup_voxels: CGA index of each voxel, UINT32_MAX when absent.
 * garrays_x: the G-Arrays X_pointer, one cell per x value of the whole axis
 * (2^bits + 1 entries): xptr[v] = number of (x, y) columns with x < v.
 * garrays_lookup: the lookup through that pointer array (same answer).
 * nn_voxels: exact NN (Eq. 7-8) of integer voxels clamped to +-2^30. */
int orc_lookup_voxels(const orc_cga* a, const int32_t* qv, uint64_t m, uint32_t* idx);
int orc_garrays_x(const orc_cga* a, uint32_t* xptr);
int orc_garrays_lookup(const orc_cga* a, const uint32_t* xptr, const int32_t* qv, uint64_t m,
                       uint32_t* idx);
int orc_nn_voxels(const orc_cga* a, const int32_t* qv, uint64_t m, uint32_t* idx,
                  uint64_t* dist2);

/* k-means of the stored voxels (Sec. V-D clustering): 8 centres seeded at
 * the bounding box's corners (corner c: max of axis a where bit a of c is
 * set), centres in 1/256 voxel (int64, 8 * 3), squared distances to them in
 * those units, ties to the lower cluster; stop after the first pass that
 * changes no label, or after max_iter (>= 1) passes; an update sets each
 * non-empty cluster's centre to (256 * sum + n / 2) / n per axis.
 * label: u entries; counts: 8; iters: passes done (0 for an empty CGA, whose
 * centres and counts are 0). */
int orc_kmeans(const orc_cga* a, uint32_t max_iter, uint8_t* label, int64_t* centres,
               uint64_t* counts, uint32_t* iters);
/* mv[c] = ref[c] - pred[c] per axis (1/256 voxel), 0 where either is empty. */
int orc_motion_vectors(const int64_t* ref_centres, const uint64_t* ref_counts,
                       const int64_t* pred_centres, const uint64_t* pred_counts, int64_t* mv);
/* out[3i + a] = voxel_a + floor((mv[label][a] + 128) / 256), u * 3 int32. */
int orc_reconstruct(const orc_cga* a, const uint8_t* label, const int64_t* mv, int32_t* out);
/* Residual frame (Sec. V-D): out[i*C + c] = pred[i*C + c] - ref[idx[i]*C + c]
 * (int16), or pred[i*C + c] when idx[i] >= u_ref (no correspondence). */
int orc_residual(const uint8_t* pred, uint64_t u_pred, const uint8_t* ref, uint64_t u_ref,
                 const uint32_t* idx, uint32_t channels, int16_t* out);

#ifdef __cplusplus
}
#endif
#endif
