/*
 * CPU oracle for the CGA hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C++17.  It is the yardstick for the CUDA
 * library and shares nothing with it.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  Build flags: -O2 -ffp-contract=off (no
 * fused multiply-add other than the explicit std::fmaf calls below).
 *
 * Readings of the paper where it is silent (each also listed in the design
 * notes of the repository):
 *  - Quantization (the paper gives no formula; Sec. II-E-2-a asks for a
 *    bounding box that includes all points, Sec. VI-C uses QP = bits per axis):
 *    q = floorf(fmaf(p, scale, offset)), clamped in float to [0, 2^b - 1].
 *  - Rigid transform before merging (Sec. II-A, views brought to a common
 *    frame): p' = R p + t with the fixed nesting
 *    p'_r = fmaf(R[r][0], x, fmaf(R[r][1], y, fmaf(R[r][2], z, t[r]))).
 *  - Arrays are sorted ascending at every level (x, then y, then z), duplicate
 *    voxels are stored once (Sec. V), X_pointer is indexed by rank in
 *    X_index (h + 1 entries), and a Y_pointer count is per (x, y) column.
 *  - NN: query voxel not clamped to the grid (only to +-2^30), squared integer
 *    distance, ties broken by the smaller key (Eq. 8 allows a set).
 *
 * Parity pinned: see the not-gpu tests (hand fixtures, closed forms,
 * invariants, independent numpy routines, exhaustive search).
 */
#include "cga_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <iterator>
#include <vector>

namespace {

bool finite(float v) { return std::isfinite(v); }

// Sec. II-E-2-a / Sec. VI-C reading: one float per axis, clamped to the box.
uint32_t quantize_axis(float v, float scale, float offset, uint32_t bits) {
  float f = std::floor(std::fmaf(v, scale, offset));
  const float hi = (float)((1u << bits) - 1u);
  if (f < 0.0f) f = 0.0f;
  if (f > hi) f = hi;
  return (uint32_t)f;
}

// NN query reading: same floor(fma), clamped only to +-2^30.
int64_t quantize_query_axis(float v, float scale, float offset) {
  float f = std::floor(std::fmaf(v, scale, offset));
  const float lim = 1073741824.0f;  // 2^30
  if (f < -lim) f = -lim;
  if (f > lim) f = lim;
  return (int64_t)f;
}

uint64_t make_key(uint64_t x, uint64_t y, uint64_t z, uint32_t bits) {
  return (x << (2 * bits)) | (y << bits) | z;
}

uint32_t key_x(uint64_t k, uint32_t b) { return (uint32_t)(k >> (2 * b)); }
uint32_t key_y(uint64_t k, uint32_t b) {
  return (uint32_t)((k >> b) & ((1ull << b) - 1));
}
uint32_t key_z(uint64_t k, uint32_t b) {
  return (uint32_t)(k & ((1ull << b) - 1));
}

bool bits_ok(uint32_t bits) { return bits >= 1 && bits <= 16; }

// Largest r with r*r <= v.
uint64_t isqrt_u64(uint64_t v) {
  uint64_t r = (uint64_t)std::sqrt((long double)v);
  while (r > 0 && r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

}  // namespace

extern "C" {

int orc_grid_from_box(const float lo[3], float extent, uint32_t bits,
                      float* scale, float offset[3]) {
  if (!bits_ok(bits) || !(extent > 0.0f) || !finite(extent)) {
    return ORC_ERR_INVALID_ARG;
  }
  const float s = (float)(1u << bits) / extent;
  if (!finite(s)) return ORC_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a) {
    if (!finite(lo[a])) return ORC_ERR_INVALID_ARG;
    const float prod = lo[a] * s;
    offset[a] = -prod;
  }
  *scale = s;
  return ORC_OK;
}

int orc_quantize(const float* xyz, uint64_t n, uint32_t bits, float scale,
                 const float offset[3], const float* xform12, uint64_t* keys) {
  if (!bits_ok(bits)) return ORC_ERR_INVALID_ARG;
  int status = ORC_OK;
  for (uint64_t i = 0; i < n; ++i) {
    float p[3] = {xyz[3 * i + 0], xyz[3 * i + 1], xyz[3 * i + 2]};
    bool ok = finite(p[0]) && finite(p[1]) && finite(p[2]);
    if (ok && xform12 != nullptr) {
      const float* R = xform12;
      const float* t = xform12 + 9;
      float r[3];
      for (int row = 0; row < 3; ++row) {
        r[row] = std::fmaf(R[3 * row + 0], p[0],
                           std::fmaf(R[3 * row + 1], p[1],
                                     std::fmaf(R[3 * row + 2], p[2], t[row])));
      }
      p[0] = r[0];
      p[1] = r[1];
      p[2] = r[2];
      ok = finite(p[0]) && finite(p[1]) && finite(p[2]);
    }
    if (!ok) {
      status = ORC_ERR_NONFINITE;
      keys[i] = 0;
      continue;
    }
    const uint32_t x = quantize_axis(p[0], scale, offset[0], bits);
    const uint32_t y = quantize_axis(p[1], scale, offset[1], bits);
    const uint32_t z = quantize_axis(p[2], scale, offset[2], bits);
    keys[i] = make_key(x, y, z, bits);
  }
  return status;
}

// Sec. V: Z_index holds the z of every stored point; Y_index the y of every
// distinct (x, y) column with Y_pointer[0] = 0 and Y_pointer[i+1] =
// Y_pointer[i] + (points in column i); X_index every distinct x with
// X_pointer[0] = 0 and X_pointer[i+1] = X_pointer[i] + (distinct y at that x).
int orc_from_sorted_keys(const uint64_t* keys, uint64_t u, uint32_t bits,
                         orc_cga* out) {
  if (!bits_ok(bits)) return ORC_ERR_INVALID_ARG;
  std::vector<uint32_t> col_x, col_y, col_count;
  for (uint64_t i = 0; i < u; ++i) {
    const uint32_t x = key_x(keys[i], bits), y = key_y(keys[i], bits);
    if (col_x.empty() || col_x.back() != x || col_y.back() != y) {
      col_x.push_back(x);
      col_y.push_back(y);
      col_count.push_back(0);
    }
    col_count.back() += 1;
    out->Z_index[i] = (uint16_t)key_z(keys[i], bits);
  }
  const uint64_t g = col_x.size();
  out->Y_pointer[0] = 0;
  for (uint64_t j = 0; j < g; ++j) {
    out->Y_index[j] = (uint16_t)col_y[j];
    out->Y_pointer[j + 1] = out->Y_pointer[j] + col_count[j];
  }
  std::vector<uint32_t> xs, x_count;
  for (uint64_t j = 0; j < g; ++j) {
    if (xs.empty() || xs.back() != col_x[j]) {
      xs.push_back(col_x[j]);
      x_count.push_back(0);
    }
    x_count.back() += 1;
  }
  const uint64_t h = xs.size();
  out->X_pointer[0] = 0;
  for (uint64_t k = 0; k < h; ++k) {
    out->X_index[k] = (uint16_t)xs[k];
    out->X_pointer[k + 1] = out->X_pointer[k] + x_count[k];
  }
  out->bits = bits;
  out->h = h;
  out->g = g;
  out->u = u;
  return ORC_OK;
}

int orc_build(const float* xyz, uint64_t n, uint32_t bits, float scale,
              const float offset[3], const float* xform12, orc_cga* out) {
  if (!bits_ok(bits)) return ORC_ERR_INVALID_ARG;
  std::vector<uint64_t> keys(n);
  const int st = orc_quantize(xyz, n, bits, scale, offset, xform12, keys.data());
  if (st != ORC_OK) return st;
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  return orc_from_sorted_keys(keys.data(), keys.size(), bits, out);
}

// Nested walk X -> Y -> Z (Sec. V-A access order).
int orc_decode_keys(const orc_cga* a, uint64_t* keys) {
  uint64_t p = 0;
  for (uint64_t i = 0; i < a->h; ++i) {
    for (uint32_t j = a->X_pointer[i]; j < a->X_pointer[i + 1]; ++j) {
      for (uint32_t k = a->Y_pointer[j]; k < a->Y_pointer[j + 1]; ++k) {
        keys[p++] = make_key(a->X_index[i], a->Y_index[j], a->Z_index[k],
                             a->bits);
      }
    }
  }
  return p == a->u ? ORC_OK : ORC_ERR_INVALID_ARG;
}

int orc_decode(const orc_cga* a, uint32_t* xyz) {
  uint64_t p = 0;
  for (uint64_t i = 0; i < a->h; ++i) {
    for (uint32_t j = a->X_pointer[i]; j < a->X_pointer[i + 1]; ++j) {
      for (uint32_t k = a->Y_pointer[j]; k < a->Y_pointer[j + 1]; ++k) {
        xyz[3 * p + 0] = a->X_index[i];
        xyz[3 * p + 1] = a->Y_index[j];
        xyz[3 * p + 2] = a->Z_index[k];
        ++p;
      }
    }
  }
  return p == a->u ? ORC_OK : ORC_ERR_INVALID_ARG;
}

// Sec. V-A lookup: find x in X_index, then y among Y_index[X_pointer[i] ..
// X_pointer[i+1]), then z among Z_index[Y_pointer[k] .. Y_pointer[k+1]).
int64_t orc_lookup(const orc_cga* a, uint32_t x, uint32_t y, uint32_t z) {
  const uint16_t* xb = a->X_index;
  const uint16_t* xe = a->X_index + a->h;
  const uint16_t* xi = std::lower_bound(xb, xe, (uint16_t)x);
  if (x > 0xFFFFu || xi == xe || *xi != x) return -1;
  const uint64_t i = (uint64_t)(xi - xb);
  const uint16_t* yb = a->Y_index + a->X_pointer[i];
  const uint16_t* ye = a->Y_index + a->X_pointer[i + 1];
  const uint16_t* yi = std::lower_bound(yb, ye, (uint16_t)y);
  if (y > 0xFFFFu || yi == ye || *yi != y) return -1;
  const uint64_t k = (uint64_t)(yi - a->Y_index);
  const uint16_t* zb = a->Z_index + a->Y_pointer[k];
  const uint16_t* ze = a->Z_index + a->Y_pointer[k + 1];
  const uint16_t* zi = std::lower_bound(zb, ze, (uint16_t)z);
  if (z > 0xFFFFu || zi == ze || *zi != z) return -1;
  return (int64_t)(zi - a->Z_index);
}

// Eq. 1: the merged cloud is the set union of the voxels of both inputs.
int orc_merge(const orc_cga* a, const orc_cga* b, orc_cga* out) {
  if (a->bits != b->bits) return ORC_ERR_INVALID_ARG;
  std::vector<uint64_t> ka(a->u), kb(b->u), ko;
  if (orc_decode_keys(a, ka.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  if (orc_decode_keys(b, kb.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  ko.reserve(ka.size() + kb.size());
  std::set_union(ka.begin(), ka.end(), kb.begin(), kb.end(),
                 std::back_inserter(ko));
  return orc_from_sorted_keys(ko.data(), ko.size(), a->bits, out);
}

// Eq. 3 with m_x = m_y = 1 drops one axis; the projected cloud is the set of
// distinct 2D voxels, stored as a 2-level CGA (U_pointer recurrence as
// X_pointer in Sec. V).
int orc_project(const orc_cga* a, int plane, orc_cga2d* out) {
  if (plane < 0 || plane > 2) return ORC_ERR_INVALID_ARG;
  const uint32_t b = a->bits;
  std::vector<uint32_t> xyz(a->u * 3);
  if (orc_decode(a, xyz.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  std::vector<uint32_t> k2(a->u);
  for (uint64_t i = 0; i < a->u; ++i) {
    const uint32_t x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    uint32_t u = 0, v = 0;
    if (plane == 0) { u = x; v = y; }
    if (plane == 1) { u = x; v = z; }
    if (plane == 2) { u = y; v = z; }
    k2[i] = (u << b) | v;
  }
  std::sort(k2.begin(), k2.end());
  k2.erase(std::unique(k2.begin(), k2.end()), k2.end());
  std::vector<uint32_t> us, ucount;
  for (uint64_t j = 0; j < k2.size(); ++j) {
    const uint32_t u = k2[j] >> b;
    if (us.empty() || us.back() != u) {
      us.push_back(u);
      ucount.push_back(0);
    }
    ucount.back() += 1;
    out->V_index[j] = (uint16_t)(k2[j] & ((1u << b) - 1u));
  }
  out->U_pointer[0] = 0;
  for (uint64_t i = 0; i < us.size(); ++i) {
    out->U_index[i] = (uint16_t)us[i];
    out->U_pointer[i + 1] = out->U_pointer[i] + ucount[i];
  }
  out->bits = b;
  out->h = us.size();
  out->g = k2.size();
  return ORC_OK;
}

namespace {

struct Query {
  bool valid;
  int64_t q[3];
};

Query make_query(const float* p, float scale, const float offset[3]) {
  Query r{};
  r.valid = finite(p[0]) && finite(p[1]) && finite(p[2]);
  if (!r.valid) return r;
  for (int a = 0; a < 3; ++a) r.q[a] = quantize_query_axis(p[a], scale, offset[a]);
  return r;
}

uint64_t sq(int64_t d) { return (uint64_t)(d * d); }

// Eq. 7 squared, in integer voxel units.
uint64_t dist2(const int64_t q[3], uint32_t x, uint32_t y, uint32_t z) {
  return sq(q[0] - (int64_t)x) + sq(q[1] - (int64_t)y) + sq(q[2] - (int64_t)z);
}

// Lexicographic (distance, key) order: Eq. 8 with the smaller-key tie rule.
struct Best {
  uint64_t d2 = UINT64_MAX;
  uint64_t key = UINT64_MAX;
  uint64_t idx = UINT64_MAX;
  void offer(uint64_t d, uint64_t k, uint64_t i) {
    if (d < d2 || (d == d2 && k < key)) {
      d2 = d;
      key = k;
      idx = i;
    }
  }
};

// Index into a sorted uint16 list of the element nearest to v (ties: the
// smaller element).
uint64_t nearest_in(const uint16_t* lo, const uint16_t* hi, int64_t v) {
  const int64_t c = std::min<int64_t>(std::max<int64_t>(v, 0), 0xFFFF);
  const uint16_t* it = std::lower_bound(lo, hi, (uint16_t)c);
  if (it == hi) return (uint64_t)(hi - lo) - 1;
  if (it == lo) return 0;
  const int64_t above = (int64_t)*it - v, below = v - (int64_t)*(it - 1);
  return (below <= above) ? (uint64_t)(it - 1 - lo) : (uint64_t)(it - lo);
}

// [first, last) index range of a sorted uint16 list within [lo_v, hi_v].
void window_in(const uint16_t* lo, const uint16_t* hi, int64_t lo_v,
               int64_t hi_v, uint64_t* first, uint64_t* last) {
  if (hi_v < 0 || lo_v > 0xFFFF || lo_v > hi_v) {
    *first = *last = 0;
    return;
  }
  const uint16_t a = (uint16_t)std::max<int64_t>(lo_v, 0);
  const uint16_t b = (uint16_t)std::min<int64_t>(hi_v, 0xFFFF);
  *first = (uint64_t)(std::lower_bound(lo, hi, a) - lo);
  *last = (uint64_t)(std::upper_bound(lo, hi, b) - lo);
}

}  // namespace

int orc_query_voxels(const float* q, uint64_t m, float scale, const float offset[3],
                     int64_t* out, uint8_t* valid) {
  for (uint64_t j = 0; j < m; ++j) {
    const Query Q = make_query(q + 3 * j, scale, offset);
    valid[j] = Q.valid ? 1 : 0;
    for (int a = 0; a < 3; ++a) out[3 * j + a] = Q.valid ? Q.q[a] : 0;
  }
  return ORC_OK;
}

// Eq. 7-8 by exhaustive search.
int orc_nn_brute(const orc_cga* a, float scale, const float offset[3],
                 const float* q, uint64_t m, uint32_t* idx, uint64_t* dist2_out) {
  std::vector<uint64_t> keys(a->u);
  if (orc_decode_keys(a, keys.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  const uint32_t b = a->bits;
  for (uint64_t j = 0; j < m; ++j) {
    const Query Q = make_query(q + 3 * j, scale, offset);
    Best best;
    if (Q.valid) {
      for (uint64_t i = 0; i < a->u; ++i) {
        best.offer(dist2(Q.q, key_x(keys[i], b), key_y(keys[i], b),
                         key_z(keys[i], b)),
                   keys[i], i);
      }
    }
    idx[j] = best.idx == UINT64_MAX ? UINT32_MAX : (uint32_t)best.idx;
    dist2_out[j] = best.d2;
  }
  return ORC_OK;
}

// Sec. V-C procedure.
int orc_nn_window(const orc_cga* a, float scale, const float offset[3],
                  const float* q, uint64_t m, uint32_t* idx, uint64_t* dist2_out) {
  const uint32_t b = a->bits;
  for (uint64_t j = 0; j < m; ++j) {
    const Query Q = make_query(q + 3 * j, scale, offset);
    idx[j] = UINT32_MAX;
    dist2_out[j] = UINT64_MAX;
    if (!Q.valid || a->u == 0) continue;
    const int64_t qx = Q.q[0], qy = Q.q[1], qz = Q.q[2];
    const int64_t top = (int64_t)((1u << b) - 1u);
    // Step 1: a stored voxel equal to the query voxel.
    if (qx >= 0 && qy >= 0 && qz >= 0 && qx <= top && qy <= top && qz <= top) {
      const int64_t hit = orc_lookup(a, (uint32_t)qx, (uint32_t)qy, (uint32_t)qz);
      if (hit >= 0) {
        idx[j] = (uint32_t)hit;
        dist2_out[j] = 0;
        continue;
      }
    }
    // Step 2: nearest x, then nearest y at that x, then nearest z in that
    // column; its distance is the search bound epsilon.
    const uint64_t xi = nearest_in(a->X_index, a->X_index + a->h, qx);
    const uint32_t y0 = a->X_pointer[xi], y1 = a->X_pointer[xi + 1];
    const uint64_t yi = y0 + nearest_in(a->Y_index + y0, a->Y_index + y1, qy);
    const uint32_t z0 = a->Y_pointer[yi], z1 = a->Y_pointer[yi + 1];
    const uint64_t zi = z0 + nearest_in(a->Z_index + z0, a->Z_index + z1, qz);
    const uint64_t eps2 = dist2(Q.q, a->X_index[xi], a->Y_index[yi], a->Z_index[zi]);
    const int64_t r = (int64_t)isqrt_u64(eps2);
    // Step 3: every voxel whose x, y and z each lie within epsilon of the
    // query is a candidate; keep the nearest.
    Best best;
    uint64_t xf, xl;
    window_in(a->X_index, a->X_index + a->h, qx - r, qx + r, &xf, &xl);
    for (uint64_t i = xf; i < xl; ++i) {
      const uint32_t ys = a->X_pointer[i], ye = a->X_pointer[i + 1];
      uint64_t yf, yl;
      window_in(a->Y_index + ys, a->Y_index + ye, qy - r, qy + r, &yf, &yl);
      for (uint64_t k = ys + yf; k < ys + yl; ++k) {
        const uint32_t zs = a->Y_pointer[k], ze = a->Y_pointer[k + 1];
        uint64_t zf, zl;
        window_in(a->Z_index + zs, a->Z_index + ze, qz - r, qz + r, &zf, &zl);
        for (uint64_t p = zs + zf; p < zs + zl; ++p) {
          const uint32_t x = a->X_index[i], y = a->Y_index[k], z = a->Z_index[p];
          best.offer(dist2(Q.q, x, y, z), make_key(x, y, z, b), p);
        }
      }
    }
    idx[j] = (uint32_t)best.idx;
    dist2_out[j] = best.d2;
  }
  return ORC_OK;
}

// Sec. V Value array.  Duplicate points of one voxel: Sec. III-B averages the
// attributes of the points merged into one box (pcdownsample); the other
// policy keeps the first point's.  Pairs (key, input index) sorted by key,
// then by index, give each voxel's points in input order.
int orc_build_values(const float* xyz, const uint8_t* attr, uint32_t channels, uint64_t n,
                     uint32_t bits, float scale, const float offset[3], const float* xform12,
                     int policy, orc_cga* out, uint8_t* values) {
  if (!bits_ok(bits) || channels < 1 || channels > 4) return ORC_ERR_INVALID_ARG;
  if (policy != ORC_VALUE_AVERAGE && policy != ORC_VALUE_FIRST) return ORC_ERR_INVALID_ARG;
  std::vector<uint64_t> keys(n);
  const int st = orc_quantize(xyz, n, bits, scale, offset, xform12, keys.data());
  if (st != ORC_OK) return st;
  std::vector<std::pair<uint64_t, uint64_t>> kp(n);
  for (uint64_t i = 0; i < n; ++i) kp[i] = {keys[i], i};
  std::sort(kp.begin(), kp.end());
  std::vector<uint64_t> ukeys;
  uint64_t i = 0;
  while (i < n) {
    uint64_t j = i;
    while (j < n && kp[j].first == kp[i].first) ++j;
    const uint64_t p = ukeys.size();
    for (uint32_t c = 0; c < channels; ++c) {
      if (policy == ORC_VALUE_FIRST) {
        values[p * channels + c] = attr[kp[i].second * channels + c];
      } else {
        uint64_t sum = 0;
        for (uint64_t k = i; k < j; ++k) sum += attr[kp[k].second * channels + c];
        const uint64_t cnt = j - i;
        values[p * channels + c] = (uint8_t)((sum + cnt / 2) / cnt);
      }
    }
    ukeys.push_back(kp[i].first);
    i = j;
  }
  return orc_from_sorted_keys(ukeys.data(), ukeys.size(), bits, out);
}

// Eq. 1 as a sorted union; a voxel in both inputs takes the base's (a's)
// attributes or the average of the two (Sec. II-A).
int orc_merge_values(const orc_cga* a, const uint8_t* va, const orc_cga* b, const uint8_t* vb,
                     uint32_t channels, int policy, orc_cga* out, uint8_t* values) {
  if (a->bits != b->bits || channels < 1 || channels > 4) return ORC_ERR_INVALID_ARG;
  if (policy != ORC_MERGE_BASE && policy != ORC_MERGE_AVERAGE) return ORC_ERR_INVALID_ARG;
  std::vector<uint64_t> ka(a->u), kb(b->u), ko;
  if (orc_decode_keys(a, ka.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  if (orc_decode_keys(b, kb.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  uint64_t i = 0, j = 0;
  while (i < ka.size() || j < kb.size()) {
    const uint64_t p = ko.size();
    const bool takeA = j == kb.size() || (i < ka.size() && ka[i] <= kb[j]);
    const bool both = i < ka.size() && j < kb.size() && ka[i] == kb[j];
    for (uint32_t c = 0; c < channels; ++c) {
      uint32_t v;
      if (both) {
        v = policy == ORC_MERGE_BASE ? va[i * channels + c]
                                     : (va[i * channels + c] + vb[j * channels + c] + 1u) / 2u;
      } else {
        v = takeA ? va[i * channels + c] : vb[j * channels + c];
      }
      values[p * channels + c] = (uint8_t)v;
    }
    ko.push_back(takeA ? ka[i] : kb[j]);
    if (both) {
      ++i;
      ++j;
    } else if (takeA) {
      ++i;
    } else {
      ++j;
    }
  }
  return orc_from_sorted_keys(ko.data(), ko.size(), a->bits, out);
}

// Eq. 6 (rotation about y) then Eq. 5 (perspective divide onto the plane at
// D); a pixel keeps its nearest voxel (a z-buffer), ties to the smaller index.
int orc_perspective(const orc_cga* a, const float eye[3], float cos_t, float sin_t, float D,
                    uint32_t W, uint32_t H, uint32_t* index, float* depth) {
  if (W == 0 || H == 0 || !(D > 0.0f)) return ORC_ERR_INVALID_ARG;
  const uint64_t npix = (uint64_t)W * H;
  for (uint64_t i = 0; i < npix; ++i) {
    index[i] = 0xffffffffu;
    depth[i] = INFINITY;
  }
  std::vector<uint32_t> xyz(a->u * 3);
  if (orc_decode(a, xyz.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  const float half_w = (float)W * 0.5f, half_h = (float)H * 0.5f;
  const float neg_sin = -sin_t;
  for (uint64_t p = 0; p < a->u; ++p) {
    const float sx = (float)xyz[3 * p] - eye[0];
    const float sy = (float)xyz[3 * p + 1] - eye[1];
    const float sz = (float)xyz[3 * p + 2] - eye[2];
    const float m1 = neg_sin * sz;
    const float xr = std::fmaf(cos_t, sx, m1);
    const float m2 = cos_t * sz;
    const float zr = std::fmaf(sin_t, sx, m2);
    if (!(zr > 0.0f)) continue;
    const float nx = D * xr, ny = D * sy;
    const float px = nx / zr, py = ny / zr;
    const float fu = std::floor(px + half_w), fv = std::floor(py + half_h);
    if (!(fu >= 0.0f && fu < (float)W && fv >= 0.0f && fv < (float)H)) continue;
    const uint64_t pix = (uint64_t)fv * W + (uint64_t)fu;
    if (zr < depth[pix] || (zr == depth[pix] && p < index[pix])) {
      depth[pix] = zr;
      index[pix] = (uint32_t)p;
    }
  }
  return ORC_OK;
}

// Radius search by exhaustive scan in CGA order: every voxel within the
// squared radius, ascending index.
int orc_radius_count(const orc_cga* a, float scale, const float offset[3], const float* q,
                     uint64_t m, uint64_t r2, uint64_t* counts) {
  std::vector<uint64_t> keys(a->u);
  if (orc_decode_keys(a, keys.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  const uint32_t b = a->bits;
  for (uint64_t j = 0; j < m; ++j) {
    const Query Q = make_query(q + 3 * j, scale, offset);
    uint64_t c = 0;
    if (Q.valid) {
      for (uint64_t i = 0; i < a->u; ++i) {
        if (dist2(Q.q, key_x(keys[i], b), key_y(keys[i], b), key_z(keys[i], b)) <= r2) ++c;
      }
    }
    counts[j] = c;
  }
  return ORC_OK;
}

int orc_radius_fill(const orc_cga* a, float scale, const float offset[3], const float* q,
                    uint64_t m, uint64_t r2, const uint64_t* offsets, uint32_t* idx,
                    uint64_t* dist2_out) {
  std::vector<uint64_t> keys(a->u);
  if (orc_decode_keys(a, keys.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  const uint32_t b = a->bits;
  for (uint64_t j = 0; j < m; ++j) {
    const Query Q = make_query(q + 3 * j, scale, offset);
    if (!Q.valid) continue;
    uint64_t o = offsets[j];
    for (uint64_t i = 0; i < a->u; ++i) {
      const uint64_t d = dist2(Q.q, key_x(keys[i], b), key_y(keys[i], b), key_z(keys[i], b));
      if (d <= r2) {
        idx[o] = (uint32_t)i;
        dist2_out[o] = d;
        ++o;
      }
    }
  }
  return ORC_OK;
}

// k nearest by exhaustive search: the k least (distance^2, key) pairs.
int orc_knn(const orc_cga* a, float scale, const float offset[3], const float* q, uint64_t m,
            uint32_t k, uint32_t* idx, uint64_t* dist2_out) {
  if (k == 0) return ORC_ERR_INVALID_ARG;
  std::vector<uint64_t> keys(a->u);
  if (orc_decode_keys(a, keys.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  const uint32_t b = a->bits;
  std::vector<std::pair<uint64_t, uint64_t>> cand(a->u);  // (distance^2, index); index order = key order
  for (uint64_t j = 0; j < m; ++j) {
    const Query Q = make_query(q + 3 * j, scale, offset);
    uint64_t n = 0;
    if (Q.valid) {
      for (uint64_t i = 0; i < a->u; ++i) {
        cand[i] = {dist2(Q.q, key_x(keys[i], b), key_y(keys[i], b), key_z(keys[i], b)), i};
      }
      n = a->u;
    }
    const uint64_t take = std::min<uint64_t>(k, n);
    std::partial_sort(cand.begin(), cand.begin() + take, cand.begin() + n);
    for (uint32_t t = 0; t < k; ++t) {
      idx[j * k + t] = t < take ? (uint32_t)cand[t].second : UINT32_MAX;
      dist2_out[j * k + t] = t < take ? cand[t].first : UINT64_MAX;
    }
  }
  return ORC_OK;
}

// ---- Compression pieces (Sec. V-D) and G-Arrays (Sec. V) ----------------

// Voxel query lookup: each int32 voxel (any value) by the Sec. V-A lookup.
int orc_lookup_voxels(const orc_cga* a, const int32_t* qv, uint64_t m, uint32_t* idx) {
  for (uint64_t j = 0; j < m; ++j) {
    const int32_t x = qv[3 * j], y = qv[3 * j + 1], z = qv[3 * j + 2];
    int64_t r = -1;
    if (x >= 0 && y >= 0 && z >= 0 && x <= 0xFFFF && y <= 0xFFFF && z <= 0xFFFF) {
      r = orc_lookup(a, (uint32_t)x, (uint32_t)y, (uint32_t)z);
    }
    idx[j] = r < 0 ? UINT32_MAX : (uint32_t)r;
  }
  return ORC_OK;
}

// G-Arrays X_pointer (Sec. V, the G-Arrays form): one cell per x value of
// the whole axis, xptr[v] = the number of (x, y) columns with x < v, so the
// columns of x = v are [xptr[v], xptr[v + 1]) and an absent x owns none.
int orc_garrays_x(const orc_cga* a, uint32_t* xptr) {
  const uint64_t side = 1ull << a->bits;
  std::vector<uint64_t> cols(side, 0);
  for (uint64_t i = 0; i < a->h; ++i) cols[a->X_index[i]] = a->X_pointer[i + 1] - a->X_pointer[i];
  uint64_t run = 0;
  for (uint64_t v = 0; v < side; ++v) {
    xptr[v] = (uint32_t)run;
    run += cols[v];
  }
  xptr[side] = (uint32_t)run;
  return run == a->g ? ORC_OK : ORC_ERR_INVALID_ARG;
}

// The same lookup through the G-Arrays X_pointer: the x value indexes the
// pointer array directly, then y and z are searched as in Sec. V-A.
int orc_garrays_lookup(const orc_cga* a, const uint32_t* xptr, const int32_t* qv, uint64_t m,
                       uint32_t* idx) {
  const int64_t side = 1ll << a->bits;
  for (uint64_t j = 0; j < m; ++j) {
    const int64_t x = qv[3 * j], y = qv[3 * j + 1], z = qv[3 * j + 2];
    idx[j] = UINT32_MAX;
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) continue;
    const uint16_t* yb = a->Y_index + xptr[x];
    const uint16_t* ye = a->Y_index + xptr[x + 1];
    const uint16_t* yi = std::lower_bound(yb, ye, (uint16_t)y);
    if (yi == ye || *yi != y) continue;
    const uint64_t k = (uint64_t)(yi - a->Y_index);
    const uint16_t* zb = a->Z_index + a->Y_pointer[k];
    const uint16_t* ze = a->Z_index + a->Y_pointer[k + 1];
    const uint16_t* zi = std::lower_bound(zb, ze, (uint16_t)z);
    if (zi == ze || *zi != z) continue;
    idx[j] = (uint32_t)(zi - a->Z_index);
  }
  return ORC_OK;
}

// Eq. 7-8 by exhaustive search for integer query voxels (clamped to
// [-2^30, 2^30] like quantized queries).
int orc_nn_voxels(const orc_cga* a, const int32_t* qv, uint64_t m, uint32_t* idx,
                  uint64_t* dist2_out) {
  std::vector<uint64_t> keys(a->u);
  if (orc_decode_keys(a, keys.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  const uint32_t b = a->bits;
  const int64_t lim = 1ll << 30;
  for (uint64_t j = 0; j < m; ++j) {
    int64_t q[3];
    for (int c = 0; c < 3; ++c) q[c] = std::min(std::max((int64_t)qv[3 * j + c], -lim), lim);
    Best best;
    for (uint64_t i = 0; i < a->u; ++i) {
      best.offer(dist2(q, key_x(keys[i], b), key_y(keys[i], b), key_z(keys[i], b)), keys[i], i);
    }
    idx[j] = best.idx == UINT64_MAX ? UINT32_MAX : (uint32_t)best.idx;
    dist2_out[j] = best.d2;
  }
  return ORC_OK;
}

// Sec. V-D clustering: k-means (Lloyd's iteration) of the stored voxels with
// eight centres, first placed at the corners of the frame's bounding box
// (corner c takes the maximum of axis a when bit a of c is set, else the
// minimum).  Centres are kept in 1/256 voxel units.  Each pass assigns every
// voxel to the centre of least squared distance (ties: the lower cluster);
// when a pass changes no label the iteration has converged and stops, else
// each non-empty cluster's centre becomes its members' mean, rounded half up
// to 1/256 (an empty cluster keeps its centre).  At most max_iter passes.
int orc_kmeans(const orc_cga* a, uint32_t max_iter, uint8_t* label, int64_t* centres,
               uint64_t* counts, uint32_t* iters) {
  if (max_iter == 0) return ORC_ERR_INVALID_ARG;
  const uint64_t u = a->u;
  std::vector<uint32_t> v(3 * u);
  if (orc_decode(a, v.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  for (int i = 0; i < 24; ++i) centres[i] = 0;
  for (int c = 0; c < 8; ++c) counts[c] = 0;
  *iters = 0;
  if (u == 0) return ORC_OK;
  uint32_t lo[3] = {UINT32_MAX, UINT32_MAX, UINT32_MAX}, hi[3] = {0, 0, 0};
  for (uint64_t i = 0; i < u; ++i) {
    for (int ax = 0; ax < 3; ++ax) {
      lo[ax] = std::min(lo[ax], v[3 * i + ax]);
      hi[ax] = std::max(hi[ax], v[3 * i + ax]);
    }
  }
  for (int c = 0; c < 8; ++c) {
    for (int ax = 0; ax < 3; ++ax) centres[3 * c + ax] = 256 * (int64_t)(((c >> ax) & 1) ? hi[ax] : lo[ax]);
  }
  std::vector<uint8_t> prev(u, 0);
  uint32_t t = 0;
  while (t < max_iter) {
    ++t;
    bool changed = false;
    for (uint64_t i = 0; i < u; ++i) {
      uint64_t best = UINT64_MAX;
      uint8_t bl = 0;
      for (int c = 0; c < 8; ++c) {
        uint64_t d = 0;
        for (int ax = 0; ax < 3; ++ax) {
          const int64_t diff = 256 * (int64_t)v[3 * i + ax] - centres[3 * c + ax];
          d += (uint64_t)(diff * diff);
        }
        if (d < best) {
          best = d;
          bl = (uint8_t)c;
        }
      }
      if (t > 1 && bl != prev[i]) changed = true;
      label[i] = bl;
    }
    if (t > 1 && !changed) break;
    uint64_t S[8][3] = {}, N[8] = {};
    for (uint64_t i = 0; i < u; ++i) {
      ++N[label[i]];
      for (int ax = 0; ax < 3; ++ax) S[label[i]][ax] += v[3 * i + ax];
      prev[i] = label[i];
    }
    for (int c = 0; c < 8; ++c) {
      if (N[c] == 0) continue;
      for (int ax = 0; ax < 3; ++ax) centres[3 * c + ax] = (int64_t)((256 * S[c][ax] + N[c] / 2) / N[c]);
    }
  }
  for (uint64_t i = 0; i < u; ++i) ++counts[label[i]];
  *iters = t;
  return ORC_OK;
}

// Sec. V-D cluster motion: the change of each cluster's centroid between the
// predicted and the reference frame, mv[c] = ref[c] - pred[c] (1/256 voxel),
// zero where either cluster is empty.
int orc_motion_vectors(const int64_t* ref_centres, const uint64_t* ref_counts,
                       const int64_t* pred_centres, const uint64_t* pred_counts, int64_t* mv) {
  for (int c = 0; c < 8; ++c) {
    for (int ax = 0; ax < 3; ++ax) {
      mv[3 * c + ax] = (ref_counts[c] > 0 && pred_counts[c] > 0)
                           ? ref_centres[3 * c + ax] - pred_centres[3 * c + ax]
                           : 0;
    }
  }
  return ORC_OK;
}

// Sec. V-D reconstructed frame: every voxel of the predicted frame moved by
// its cluster's motion vector rounded half up to whole voxels,
// r = v + floor((mv + 128) / 256) per axis (not clamped to the grid).
int orc_reconstruct(const orc_cga* a, const uint8_t* label, const int64_t* mv, int32_t* out) {
  std::vector<uint32_t> v(3 * a->u);
  if (orc_decode(a, v.data()) != ORC_OK) return ORC_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < a->u; ++i) {
    if (label[i] > 7) return ORC_ERR_INVALID_ARG;
    for (int ax = 0; ax < 3; ++ax) {
      const int64_t m = mv[3 * label[i] + ax];
      const int64_t num = m + 128;
      const int64_t fl = num >= 0 ? num / 256 : -((-num + 255) / 256);
      out[3 * i + ax] = (int32_t)((int64_t)v[3 * i + ax] + fl);
    }
  }
  return ORC_OK;
}

// Sec. V-D residual frame: for every point of the reconstructed (predicted)
// frame the difference between its attributes and those of its
// corresponding reference point, res = pred - ref[idx] per channel; a point
// without a correspondence (idx out of range) keeps its own attributes.
int orc_residual(const uint8_t* pred, uint64_t u_pred, const uint8_t* ref, uint64_t u_ref,
                 const uint32_t* idx, uint32_t channels, int16_t* out) {
  if (channels < 1 || channels > 4) return ORC_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < u_pred; ++i) {
    for (uint32_t c = 0; c < channels; ++c) {
      const int16_t p = (int16_t)pred[i * channels + c];
      out[i * channels + c] =
          idx[i] < u_ref ? (int16_t)(p - (int16_t)ref[(uint64_t)idx[i] * channels + c]) : p;
    }
  }
  return ORC_OK;
}

}  // extern "C"
