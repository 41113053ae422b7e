// C-ABI of libcga (include/cga.h): argument checks, handle and memory
// management, and the launch sequences of the kernels in k_sort.cu / k_ops.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/cga.h"
#include "cga_impl.h"

using libcga::Header;
using libcga::Levels;

struct cga {
  cga_grid grid;
  Levels lv;
  void* mem;
  cga_allocator alloc;
  bool has_alloc;
  cudaStream_t stream;
  bool view = false;  // arrays owned by a pipeline; cga_free leaves them alone
  // coarse levels for NN (cga_nn_prepare_levels): level k is the CGA of the
  // occupied cells of 2^cshift[k] voxels, with its slab index into the next
  // finer level and its own x directory (all inside cmem[k])
  uint32_t ncoarse = 0;
  void* cmem[libcga::kMaxCoarse] = {};
  Levels clv[libcga::kMaxCoarse] = {};
  uint32_t* xs[libcga::kMaxCoarse] = {};
  uint32_t cshift[libcga::kMaxCoarse] = {};
  uint32_t* cxdir[libcga::kMaxCoarse] = {};
  uint4* czr[libcga::kMaxCoarse] = {};
  uint32_t* cchild[libcga::kMaxCoarse] = {};
  // Value array (cga_build_values / cga_merge_values): channels bytes per voxel
  void* vmem = nullptr;
  uint8_t* values = nullptr;
  uint32_t channels = 0;
  // x directory of this CGA for NN (cga_nn_prepare): first X_index entry >= v
  void* xdmem = nullptr;
  uint32_t* xdir = nullptr;
  // column table of this CGA for NN (cga_nn_prepare): voxel range + z range
  void* zrmem = nullptr;
  uint4* ctab = nullptr;
  // occupancy tree for NN (cga_nn_prepare_levels with CGA_NN_TREE)
  void* tmem = nullptr;
  libcga::TreeView tree{};
};

struct cga2d {
  uint32_t bits;
  int plane;
  Levels lv;
  void* mem;
  cga_allocator alloc;
  bool has_alloc;
  cudaStream_t stream;
  bool view = false;
};

namespace libcga {
// The arrays and grid behind a handle, for entry points in other files.
void handle_parts(const cga_t* a, Levels* lv, cga_grid* g) {
  *lv = a->lv;
  *g = a->grid;
}
void nn_attach(const cga_t* a, NnSeg& seg);
void rebind_stream(cga_t* a, cga2d_t* p, cudaStream_t s) {
  if (a != nullptr) a->stream = s;
  if (p != nullptr) p->stream = s;
}
static std::atomic<uint64_t> g_launches{0};
void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace libcga

namespace {

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Default allocator: one stream-ordered memory pool per device, owned by the
// library and kept warm (freed blocks stay in the pool for reuse).
cudaMemPool_t device_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (pools[dev] == nullptr) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

void* dalloc(const cga_allocator* A, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 256;
  if (A != nullptr && A->alloc != nullptr) return A->alloc(A->ctx, bytes, s);
  void* p = nullptr;
  cudaMemPool_t pool = device_pool();
  if (pool == nullptr || cudaMallocFromPoolAsync(&p, bytes, pool, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dfree(const cga_allocator* A, bool has, void* p, cudaStream_t s) {
  if (p == nullptr) return;
  if (has && A->free != nullptr) {
    A->free(A->ctx, p, s);
    return;
  }
  if (!has) cudaFreeAsync(p, s);
}

bool grid_ok(const cga_grid* g) {
  if (g == nullptr || g->bits < 1 || g->bits > 16) return false;
  if (!std::isfinite(g->scale) || !(g->scale > 0.0f)) return false;
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(g->offset[a])) return false;
  }
  return true;
}

bool same_grid(const cga_grid& a, const cga_grid& b) {
  return a.bits == b.bits && std::memcmp(&a.scale, &b.scale, sizeof(float)) == 0 &&
         std::memcmp(a.offset, b.offset, sizeof(a.offset)) == 0;
}

uint64_t pow2(uint32_t e) { return e >= 63 ? ~0ull : (1ull << e); }

// Carve a Levels structure (header + arrays) out of one allocation.
size_t levels_bytes(uint64_t cap, uint64_t cap1, uint64_t cap2, int nlevels) {
  size_t b = align_up(sizeof(Header));
  b += align_up(cap * 2) + align_up(cap1 * 2) + align_up((cap1 + 1) * 4);
  if (nlevels == 3) b += align_up(cap2 * 2) + align_up((cap2 + 1) * 4);
  return b;
}

Levels levels_carve(void* base, uint32_t bits, uint64_t cap, uint64_t cap1, uint64_t cap2,
                    int nlevels) {
  char* p = static_cast<char*>(base);
  Levels lv{};
  lv.hdr = reinterpret_cast<Header*>(p);
  p += align_up(sizeof(Header));
  lv.idx0 = reinterpret_cast<uint16_t*>(p);
  p += align_up(cap * 2);
  lv.idx1 = reinterpret_cast<uint16_t*>(p);
  p += align_up(cap1 * 2);
  lv.ptr1 = reinterpret_cast<uint32_t*>(p);
  p += align_up((cap1 + 1) * 4);
  if (nlevels == 3) {
    lv.idx2 = reinterpret_cast<uint16_t*>(p);
    p += align_up(cap2 * 2);
    lv.ptr2 = reinterpret_cast<uint32_t*>(p);
  }
  lv.bits = bits;
  lv.nlevels = (uint32_t)nlevels;
  lv.cap = cap;
  lv.cap1 = cap1;
  lv.cap2 = nlevels == 3 ? cap2 : 0;
  return lv;
}

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return CGA_OK;
  cudaGetLastError();
  return CGA_ERR_CUDA;
}

int err_from_bits(uint32_t bits) {
  if (bits & libcga::kErrNonfinite) return CGA_ERR_NONFINITE;
  if (bits & libcga::kErrTimeout) return CGA_ERR_TIMEOUT;
  if (bits) return CGA_ERR_INTERNAL;
  return CGA_OK;
}

int read_header(const Levels& lv, cudaStream_t s, Header* h) {
  cudaError_t e = cudaMemcpyAsync(h, lv.hdr, sizeof(Header), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_rc(e);
}

cga* new_cga(const cga_grid& g, const cga_allocator* A, cudaStream_t s, uint64_t cap) {
  const uint32_t b = g.bits;
  const uint64_t cap1 = std::min<uint64_t>(cap, pow2(2 * b));
  const uint64_t cap2 = std::min<uint64_t>(cap, pow2(b));
  void* mem = dalloc(A, levels_bytes(cap, cap1, cap2, 3), s);
  if (mem == nullptr) return nullptr;
  cga* h = new (std::nothrow) cga{};
  if (h == nullptr) {
    dfree(A, A != nullptr, mem, s);
    return nullptr;
  }
  h->grid = g;
  h->lv = levels_carve(mem, b, cap, cap1, cap2, 3);
  h->mem = mem;
  h->has_alloc = A != nullptr;
  if (A != nullptr) h->alloc = *A;
  h->stream = s;
  return h;
}

void release(cga* h) {
  if (h == nullptr || h->view) return;
  for (int k = 0; k < libcga::kMaxCoarse; ++k) {
    if (h->cmem[k] != nullptr) dfree(&h->alloc, h->has_alloc, h->cmem[k], h->stream);
  }
  if (h->xdmem != nullptr) dfree(&h->alloc, h->has_alloc, h->xdmem, h->stream);
  if (h->vmem != nullptr) dfree(&h->alloc, h->has_alloc, h->vmem, h->stream);
  if (h->zrmem != nullptr) dfree(&h->alloc, h->has_alloc, h->zrmem, h->stream);
  if (h->tmem != nullptr) dfree(&h->alloc, h->has_alloc, h->tmem, h->stream);
  dfree(&h->alloc, h->has_alloc, h->mem, h->stream);
  delete h;
}

// NN searches use the coarse levels that cga_nn_prepare_levels built.
void attach_coarse(const cga* a, libcga::NnSeg& seg) {
  seg.xdir = a->xdir;
  seg.ctab = a->ctab;
  seg.tree = a->tree;
  seg.ncoarse = a->ncoarse;
  for (uint32_t k = 0; k < a->ncoarse; ++k) {
    seg.c[k] = a->clv[k];
    seg.xs[k] = a->xs[k];
    seg.shift[k] = a->cshift[k];
    seg.cxdir[k] = a->cxdir[k];
    seg.zr[k] = a->czr[k];
    seg.child[k] = a->cchild[k];
  }
}

}  // namespace

namespace libcga {
// The NN search structures prepared on a handle (x directory, column table,
// coarse levels or occupancy tree), for entry points in other files.
void nn_attach(const cga_t* a, NnSeg& seg) { attach_coarse(a, seg); }
}  // namespace libcga

extern "C" {

int cga_grid_from_box(const float lo[3], float extent, uint32_t bits, cga_grid* out) {
  if (lo == nullptr || out == nullptr || bits < 1 || bits > 16) return CGA_ERR_INVALID_ARG;
  if (!std::isfinite(extent) || !(extent > 0.0f)) return CGA_ERR_INVALID_ARG;
  const float s = (float)(1u << bits) / extent;
  if (!std::isfinite(s)) return CGA_ERR_INVALID_ARG;
  cga_grid g{};
  g.bits = bits;
  g.scale = s;
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(lo[a])) return CGA_ERR_INVALID_ARG;
    const float prod = lo[a] * s;
    g.offset[a] = -prod;
  }
  *out = g;
  return CGA_OK;
}

int cga_build(const float* d_xyz, uint64_t n, const cga_grid* g, const float* h_xform12,
              const cga_allocator* A, void* stream, cga_t** out) {
  if (out == nullptr || !grid_ok(g) || n > CGA_MAX_POINTS || (n > 0 && d_xyz == nullptr)) {
    return CGA_ERR_INVALID_ARG;
  }
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cga* h = new_cga(*g, A, s, n);
  if (h == nullptr) return CGA_ERR_OOM;

  libcga::SortSeg seg{};
  seg.xyz = d_xyz;
  seg.scale = g->scale;
  for (int a = 0; a < 3; ++a) seg.off[a] = g->offset[a];
  if (h_xform12 != nullptr) {
    std::memcpy(seg.X, h_xform12, sizeof(seg.X));
    seg.has_x = 1;
  }
  seg.from_cga = 0;
  seg.n_host = (uint32_t)n;
  seg.bits = g->bits;
  seg.key_bits = 3 * g->bits;
  const libcga::Tuning tu = libcga::tuning_for(g->bits, n);
  seg.passes = libcga::radix_passes(seg.key_bits, tu.radix_bits);
  seg.key_base = 0;
  seg.tile_base = 0;
  seg.num_tiles = (uint32_t)((n + libcga::kTile - 1) / libcga::kTile);
  seg.out = h->lv;
  const bool key64 = seg.key_bits > 32;
  const uint32_t tiles = seg.num_tiles;
  const uint64_t keys = (uint64_t)tiles * libcga::kTile;
  void* scratch = dalloc(A, libcga::sort_scratch_bytes(keys, tiles, 1, key64, tu.radix_bits), s);
  if (scratch == nullptr) {
    release(h);
    return CGA_ERR_OOM;
  }
  const libcga::SortScratch sc = libcga::sort_scratch_carve(scratch, keys, tiles, 1, key64, tu);
  const int rc = cuda_rc(libcga::run_sort_pipeline(&seg, 1, tiles, seg.passes, key64, sc, s));
  dfree(A, A != nullptr, scratch, s);
  if (rc != CGA_OK) {
    release(h);
    return rc;
  }
  *out = h;
  return CGA_OK;
}

int cga_merge(const cga_t* a, const cga_t* b, const cga_allocator* A, void* stream,
              cga_t** out) {
  if (a == nullptr || b == nullptr || out == nullptr) return CGA_ERR_INVALID_ARG;
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  if (!same_grid(a->grid, b->grid)) return CGA_ERR_GRID_MISMATCH;
  const uint32_t bits = a->grid.bits;
  const uint64_t cap = std::min<uint64_t>(a->lv.cap + b->lv.cap, pow2(3 * bits));
  if (cap > CGA_MAX_POINTS) return CGA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cga* h = new_cga(a->grid, A, s, cap);
  if (h == nullptr) return CGA_ERR_OOM;
  libcga::MergePair P{};
  P.a = a->lv;
  P.b = b->lv;
  P.out = h->lv;
  P.spl_base = 0;
  const uint32_t half = libcga::tuning_for(bits, a->lv.cap + b->lv.cap).merge_half;
  P.spl_a = libcga::merge_splitters(a->lv.cap, half);
  P.spl_b = libcga::merge_splitters(b->lv.cap, half);
  P.tile_base = 0;
  P.num_tiles = P.spl_a + P.spl_b + 1;
  const uint32_t total_spl = P.spl_a + P.spl_b;
  void* scratch = dalloc(A, libcga::merge_scratch_bytes(total_spl, P.num_tiles, 1), s);
  if (scratch == nullptr) {
    release(h);
    return CGA_ERR_OOM;
  }
  const libcga::MergeScratch sc =
      libcga::merge_scratch_carve(scratch, total_spl, P.num_tiles, 1, half);
  const int rc = cuda_rc(libcga::run_merge(&P, 1, total_spl, P.num_tiles, sc, s));
  dfree(A, A != nullptr, scratch, s);
  if (rc != CGA_OK) {
    release(h);
    return rc;
  }
  *out = h;
  return CGA_OK;
}

int cga_build_values(const float* d_xyz, const uint8_t* d_attr, uint32_t channels, uint64_t n,
                     const cga_grid* g, const float* h_xform12, int policy,
                     const cga_allocator* A, void* stream, cga_t** out) {
  if (out == nullptr || channels < 1 || channels > CGA_MAX_CHANNELS ||
      (policy != CGA_VALUE_AVERAGE && policy != CGA_VALUE_FIRST) || (n > 0 && d_attr == nullptr)) {
    return CGA_ERR_INVALID_ARG;
  }
  cga_t* h = nullptr;
  int rc = cga_build(d_xyz, n, g, h_xform12, A, stream, &h);
  if (rc != CGA_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t cap = std::max<uint64_t>(h->lv.cap, 1);
  void* vm = dalloc(A, cap * channels, s);
  void* scratch = dalloc(A, libcga::value_scratch_bytes(h->lv.cap, channels, policy), s);
  if (vm == nullptr || scratch == nullptr) {
    if (vm) dfree(A, A != nullptr, vm, s);
    if (scratch) dfree(A, A != nullptr, scratch, s);
    release(h);
    return CGA_ERR_OOM;
  }
  libcga::ValueInput in{};
  in.xyz = d_xyz;
  in.attr = d_attr;
  in.n = n;
  in.channels = channels;
  in.policy = policy;
  in.scale = g->scale;
  for (int k = 0; k < 3; ++k) in.off[k] = g->offset[k];
  if (h_xform12 != nullptr) {
    std::memcpy(in.X, h_xform12, sizeof(in.X));
    in.has_x = 1;
  }
  rc = cuda_rc(libcga::run_build_values(h->lv, in, scratch, static_cast<uint8_t*>(vm), s));
  dfree(A, A != nullptr, scratch, s);
  h->vmem = vm;
  h->values = static_cast<uint8_t*>(vm);
  h->channels = channels;
  if (rc != CGA_OK) {
    release(h);
    return rc;
  }
  *out = h;
  return CGA_OK;
}

int cga_merge_values(const cga_t* a, const cga_t* b, int policy, const cga_allocator* A,
                     void* stream, cga_t** out) {
  if (a == nullptr || b == nullptr || out == nullptr || a->values == nullptr ||
      b->values == nullptr || a->channels != b->channels ||
      (policy != CGA_MERGE_BASE && policy != CGA_MERGE_AVERAGE)) {
    return CGA_ERR_INVALID_ARG;
  }
  cga_t* m = nullptr;
  int rc = cga_merge(a, b, A, stream, &m);
  if (rc != CGA_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t C = a->channels;
  void* vm = dalloc(A, std::max<uint64_t>(m->lv.cap, 1) * C, s);
  if (vm == nullptr) {
    release(m);
    return CGA_ERR_OOM;
  }
  m->vmem = vm;
  m->values = static_cast<uint8_t*>(vm);
  m->channels = C;
  rc = cuda_rc(libcga::run_merge_values(m->lv, a->lv, b->lv, a->values, b->values, C, policy,
                                        m->values, s));
  if (rc != CGA_OK) {
    release(m);
    return rc;
  }
  *out = m;
  return CGA_OK;
}

namespace {

libcga::NnSeg nn_segment(const cga_t* a, const float* d_q, uint64_t m, uint32_t* d_idx,
                         uint64_t* d_dist2) {
  libcga::NnSeg seg{};
  seg.a = a->lv;
  seg.scale = a->grid.scale;
  for (int k = 0; k < 3; ++k) seg.off[k] = a->grid.offset[k];
  seg.q = d_q;
  seg.m = (uint32_t)m;
  seg.idx = d_idx;
  seg.d2 = reinterpret_cast<unsigned long long*>(d_dist2);
  seg.tile_base = 0;
  seg.num_tiles = (uint32_t)((m + libcga::kTile - 1) / libcga::kTile);
  attach_coarse(a, seg);
  return seg;
}

}  // namespace

namespace {

// The NN search's Morton order of a query batch (sort scratch to release
// after the kernels that read it), or none for small batches.
int query_order(const cga_t* a, const float* d_q, uint64_t m, cudaStream_t s, void** scratch,
                const unsigned long long** order) {
  *scratch = nullptr;
  *order = nullptr;
  if (m < libcga::kNnSortMin || m > libcga::kNnMaxQueries) return CGA_OK;
  const libcga::NnSeg seg = nn_segment(a, d_q, m, nullptr, nullptr);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* sc = dalloc(A, libcga::nn_scratch_bytes(seg.num_tiles, 1), s);
  if (sc == nullptr) return CGA_ERR_OOM;
  const libcga::NnTables t = libcga::nn_tables(sc, seg.num_tiles, 1);
  cudaError_t e = libcga::nn_upload_one(seg, t, s);
  if (e == cudaSuccess) e = libcga::run_nn_sort_device(1, seg.num_tiles, t, s);
  if (e != cudaSuccess) {
    dfree(A, a->has_alloc, sc, s);
    return cuda_rc(e);
  }
  *scratch = sc;
  *order = static_cast<const unsigned long long*>(t.sort.keys0);
  return CGA_OK;
}

libcga::SearchSeg search_segment(const cga_t* a, const float* d_q, uint64_t m) {
  libcga::SearchSeg sg{};
  sg.a = a->lv;
  sg.scale = a->grid.scale;
  for (int k = 0; k < 3; ++k) sg.off[k] = a->grid.offset[k];
  sg.q = d_q;
  sg.m = (uint32_t)m;
  sg.ctab = a->ctab;
  return sg;
}

}  // namespace

int cga_radius_count(const cga_t* a, const float* d_q, uint64_t m, uint64_t r2,
                     uint64_t* d_offsets, void* stream) {
  if (a == nullptr || d_offsets == nullptr || (m > 0 && d_q == nullptr) || m > CGA_MAX_POINTS ||
      r2 > CGA_MAX_RADIUS2) {
    return CGA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* scratch = dalloc(A, libcga::radius_scratch_bytes(), s);
  if (scratch == nullptr) return CGA_ERR_OOM;
  void* osc = nullptr;
  const unsigned long long* order = nullptr;
  int rc = query_order(a, d_q, m, s, &osc, &order);
  if (rc == CGA_OK) {
    rc = cuda_rc(libcga::run_radius_count(search_segment(a, d_q, m), r2, order,
                                          reinterpret_cast<unsigned long long*>(d_offsets),
                                          scratch, s));
  }
  if (osc != nullptr) dfree(A, a->has_alloc, osc, s);
  dfree(A, a->has_alloc, scratch, s);
  return rc;
}

int cga_radius_fill(const cga_t* a, const float* d_q, uint64_t m, uint64_t r2,
                    const uint64_t* d_offsets, uint32_t* d_idx, uint64_t* d_dist2,
                    void* stream) {
  if (a == nullptr || (m > 0 && (d_q == nullptr || d_offsets == nullptr)) ||
      m > CGA_MAX_POINTS || r2 > CGA_MAX_RADIUS2) {
    return CGA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* osc = nullptr;
  const unsigned long long* order = nullptr;
  int rc = query_order(a, d_q, m, s, &osc, &order);
  if (rc == CGA_OK) {
    rc = cuda_rc(libcga::run_radius_fill(
        search_segment(a, d_q, m), r2, order, reinterpret_cast<const unsigned long long*>(d_offsets),
        d_idx, reinterpret_cast<unsigned long long*>(d_dist2), s));
  }
  if (osc != nullptr) dfree(A, a->has_alloc, osc, s);
  return rc;
}

static_assert(CGA_KNN_MAX_K == libcga::kKnnMaxK, "k-NN limit");

int cga_knn(const cga_t* a, const float* d_q, uint64_t m, uint32_t k, uint32_t* d_idx,
            uint64_t* d_dist2, void* stream) {
  if (a == nullptr || k < 1 || k > CGA_KNN_MAX_K || m > CGA_MAX_POINTS ||
      (m > 0 && (d_q == nullptr || d_idx == nullptr || d_dist2 == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* osc = nullptr;
  const unsigned long long* order = nullptr;
  int rc = query_order(a, d_q, m, s, &osc, &order);
  if (rc == CGA_OK) {
    rc = cuda_rc(libcga::run_knn(search_segment(a, d_q, m), k, order, d_idx,
                                 reinterpret_cast<unsigned long long*>(d_dist2), s));
  }
  if (osc != nullptr) dfree(A, a->has_alloc, osc, s);
  return rc;
}

int cga_perspective(const cga_t* a, const float eye[3], float cos_t, float sin_t, float D,
                    uint32_t W, uint32_t H, uint32_t* d_index, float* d_depth, void* stream) {
  if (a == nullptr || eye == nullptr || d_index == nullptr || d_depth == nullptr || W == 0 ||
      H == 0 || (uint64_t)W * H > CGA_MAX_PIXELS || !(D > 0.0f) || !std::isfinite(D) ||
      !std::isfinite(cos_t) || !std::isfinite(sin_t) || !std::isfinite(eye[0]) ||
      !std::isfinite(eye[1]) || !std::isfinite(eye[2])) {
    return CGA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  const uint64_t npix = (uint64_t)W * H;
  void* zbuf = dalloc(A, npix * 8, s);
  if (zbuf == nullptr) return CGA_ERR_OOM;
  libcga::Camera cam{};
  for (int k = 0; k < 3; ++k) cam.eye[k] = eye[k];
  cam.cos_t = cos_t;
  cam.sin_t = sin_t;
  cam.D = D;
  cam.W = W;
  cam.H = H;
  const int rc = cuda_rc(libcga::run_perspective(
      a->lv, cam, static_cast<unsigned long long*>(zbuf), d_index, d_depth, s));
  dfree(A, a->has_alloc, zbuf, s);
  return rc;
}

int cga_values(const cga_t* a, const uint8_t** d_values, uint32_t* channels) {
  if (a == nullptr || d_values == nullptr || channels == nullptr) return CGA_ERR_INVALID_ARG;
  *d_values = a->values;
  *channels = a->channels;
  return CGA_OK;
}

int cga_project(const cga_t* a, int plane, const cga_allocator* A, void* stream,
                cga2d_t** out) {
  if (a == nullptr || out == nullptr || plane < CGA_PLANE_XY || plane > CGA_PLANE_YZ) {
    return CGA_ERR_INVALID_ARG;
  }
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t b = a->grid.bits;
  uint64_t cap, cap1;
  if (plane == CGA_PLANE_XY) {
    cap = a->lv.cap1;
    cap1 = a->lv.cap2;
  } else {
    cap = std::min<uint64_t>(a->lv.cap, pow2(2 * b));
    cap1 = std::min<uint64_t>(cap, pow2(b));
  }
  void* mem = dalloc(A, levels_bytes(cap, cap1, 0, 2), s);
  if (mem == nullptr) return CGA_ERR_OOM;
  cga2d* p = new (std::nothrow) cga2d{};
  if (p == nullptr) {
    dfree(A, A != nullptr, mem, s);
    return CGA_ERR_OOM;
  }
  p->bits = b;
  p->plane = plane;
  p->lv = levels_carve(mem, b, cap, cap1, 0, 2);
  p->mem = mem;
  p->has_alloc = A != nullptr;
  if (A != nullptr) p->alloc = *A;
  p->stream = s;
  int rc;
  if (plane == CGA_PLANE_XY) {
    rc = cuda_rc(libcga::run_project_xy(a->lv, p->lv, s));
  } else if (b >= libcga::kProjBitmapMinBits && b <= libcga::kProjBitmapMaxBits) {
    void* scratch = dalloc(A, libcga::project_bitmap_scratch_bytes(b), s);
    if (scratch == nullptr) {
      rc = CGA_ERR_OOM;
    } else {
      rc = cuda_rc(libcga::run_project_bitmap(a->lv, plane, p->lv, scratch, s));
      dfree(A, A != nullptr, scratch, s);
    }
  } else {
    libcga::SortSeg seg{};
    seg.src = a->lv;
    seg.plane = plane;
    seg.from_cga = 1;
    seg.bits = b;
    seg.key_bits = 2 * b;
    const libcga::Tuning tu = libcga::tuning_for(b, a->lv.cap);
    seg.passes = libcga::radix_passes(seg.key_bits, tu.radix_bits);
    seg.num_tiles = (uint32_t)((a->lv.cap + libcga::kTile - 1) / libcga::kTile);
    seg.out = p->lv;
    const uint32_t tiles = seg.num_tiles;
    const uint64_t keys = (uint64_t)tiles * libcga::kTile;
    void* scratch = dalloc(A, libcga::sort_scratch_bytes(keys, tiles, 1, false, tu.radix_bits), s);
    if (scratch == nullptr) {
      rc = CGA_ERR_OOM;
    } else {
      const libcga::SortScratch sc =
          libcga::sort_scratch_carve(scratch, keys, tiles, 1, false, tu);
      rc = cuda_rc(libcga::run_sort_pipeline(&seg, 1, tiles, seg.passes, false, sc, s));
      dfree(A, A != nullptr, scratch, s);
    }
  }
  if (rc != CGA_OK) {
    dfree(A, A != nullptr, mem, s);
    delete p;
    return rc;
  }
  *out = p;
  return CGA_OK;
}

namespace {

// One NN batch of float (d_q) or integer (d_qv) queries.
int nn_query_any(const cga_t* a, const float* d_q, const int32_t* d_qv, uint64_t m,
                 uint32_t* d_idx, uint64_t* d_dist2, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  libcga::NnSeg seg = nn_segment(a, d_q, m, d_idx, d_dist2);
  seg.qv = d_qv;
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* scratch = nullptr;
  if (m >= libcga::kNnSortMin) {
    scratch = dalloc(A, libcga::nn_scratch_bytes(seg.num_tiles, 1), s);
    if (scratch == nullptr) return CGA_ERR_OOM;
  }
  const int rc = cuda_rc(libcga::run_nn(&seg, 1, seg.num_tiles, scratch, s));
  if (scratch != nullptr) dfree(A, a->has_alloc, scratch, s);
  return rc;
}

}  // namespace

int cga_nn_query(const cga_t* a, const float* d_q, uint64_t m, uint32_t* d_idx,
                 uint64_t* d_dist2, void* stream) {
  if (a == nullptr || (m > 0 && (d_q == nullptr || d_idx == nullptr || d_dist2 == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  if (m > libcga::kNnMaxQueries) return CGA_ERR_INVALID_ARG;
  if (m == 0) return CGA_OK;
  return nn_query_any(a, d_q, nullptr, m, d_idx, d_dist2, stream);
}

int cga_nn_query_voxels(const cga_t* a, const int32_t* d_qv, uint64_t m, uint32_t* d_idx,
                        uint64_t* d_dist2, void* stream) {
  if (a == nullptr || (m > 0 && (d_qv == nullptr || d_idx == nullptr || d_dist2 == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  if (m > libcga::kNnMaxQueries) return CGA_ERR_INVALID_ARG;
  if (m == 0) return CGA_OK;
  return nn_query_any(a, nullptr, d_qv, m, d_idx, d_dist2, stream);
}

int cga_kmeans(const cga_t* a, uint32_t max_iter, uint8_t* d_label, int64_t* d_centres,
               uint64_t* d_counts, uint32_t* d_iters, void* stream) {
  if (a == nullptr || d_centres == nullptr || d_counts == nullptr || d_iters == nullptr ||
      (a->lv.cap > 0 && d_label == nullptr) || max_iter < 1 || max_iter > CGA_KMEANS_MAX_ITER) {
    return CGA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* st = dalloc(A, sizeof(libcga::KmState), s);
  if (st == nullptr) return CGA_ERR_OOM;
  const int rc = cuda_rc(libcga::run_kmeans(
      a->lv, max_iter, static_cast<libcga::KmState*>(st), d_label,
      reinterpret_cast<long long*>(d_centres), reinterpret_cast<unsigned long long*>(d_counts),
      d_iters, s));
  dfree(A, a->has_alloc, st, s);
  return rc;
}

int cga_motion_vectors(const int64_t* d_ref_centres, const uint64_t* d_ref_counts,
                       const int64_t* d_pred_centres, const uint64_t* d_pred_counts,
                       int64_t* d_mv, void* stream) {
  if (d_ref_centres == nullptr || d_ref_counts == nullptr || d_pred_centres == nullptr ||
      d_pred_counts == nullptr || d_mv == nullptr) {
    return CGA_ERR_INVALID_ARG;
  }
  return cuda_rc(libcga::run_motion(
      reinterpret_cast<const long long*>(d_ref_centres),
      reinterpret_cast<const unsigned long long*>(d_ref_counts),
      reinterpret_cast<const long long*>(d_pred_centres),
      reinterpret_cast<const unsigned long long*>(d_pred_counts),
      reinterpret_cast<long long*>(d_mv), static_cast<cudaStream_t>(stream)));
}

int cga_reconstruct(const cga_t* pred, const uint8_t* d_label, const int64_t* d_mv,
                    int32_t* d_out, void* stream) {
  if (pred == nullptr || d_mv == nullptr ||
      (pred->lv.cap > 0 && (d_label == nullptr || d_out == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  return cuda_rc(libcga::run_reconstruct(pred->lv, d_label,
                                         reinterpret_cast<const long long*>(d_mv), d_out,
                                         static_cast<cudaStream_t>(stream)));
}

int cga_residual(const uint8_t* d_pred_values, uint64_t u_pred, const uint8_t* d_ref_values,
                 uint64_t u_ref, const uint32_t* d_idx, uint32_t channels, int16_t* d_out,
                 void* stream) {
  if (channels < 1 || channels > CGA_MAX_CHANNELS || u_pred > CGA_MAX_POINTS ||
      u_ref > CGA_MAX_POINTS ||
      (u_pred > 0 && (d_pred_values == nullptr || d_idx == nullptr || d_out == nullptr)) ||
      (u_ref > 0 && d_ref_values == nullptr)) {
    return CGA_ERR_INVALID_ARG;
  }
  return cuda_rc(libcga::run_residual(d_pred_values, u_pred, d_ref_values, u_ref, d_idx, channels,
                                      d_out, static_cast<cudaStream_t>(stream)));
}

int cga_garrays_x(const cga_t* a, uint32_t* d_xptr, void* stream) {
  if (a == nullptr || d_xptr == nullptr) return CGA_ERR_INVALID_ARG;
  return cuda_rc(libcga::run_garrays_x(a->lv, d_xptr, static_cast<cudaStream_t>(stream)));
}

int cga_lookup(const cga_t* a, const int32_t* d_qv, uint64_t m, uint32_t* d_idx, void* stream) {
  if (a == nullptr || (m > 0 && (d_qv == nullptr || d_idx == nullptr)) || m > CGA_MAX_POINTS) {
    return CGA_ERR_INVALID_ARG;
  }
  return cuda_rc(libcga::run_lookup(a->lv, nullptr, d_qv, (uint32_t)m, d_idx,
                                    static_cast<cudaStream_t>(stream)));
}

int cga_garrays_lookup(const cga_t* a, const uint32_t* d_xptr, const int32_t* d_qv, uint64_t m,
                       uint32_t* d_idx, void* stream) {
  if (a == nullptr || d_xptr == nullptr || (m > 0 && (d_qv == nullptr || d_idx == nullptr)) ||
      m > CGA_MAX_POINTS) {
    return CGA_ERR_INVALID_ARG;
  }
  return cuda_rc(libcga::run_lookup(a->lv, d_xptr, d_qv, (uint32_t)m, d_idx,
                                    static_cast<cudaStream_t>(stream)));
}

namespace {

static_assert(libcga::kMaxCoarse == CGA_NN_MAX_LEVELS, "coarse level count");
constexpr size_t kChildTableMaxBytes = (size_t)512 << 20;

void drop_coarse(cga* a) {
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  for (int k = 0; k < libcga::kMaxCoarse; ++k) {
    if (a->cmem[k] != nullptr) dfree(A, a->has_alloc, a->cmem[k], a->stream);
    a->cmem[k] = nullptr;
    a->clv[k] = Levels{};
    a->xs[k] = nullptr;
    a->cxdir[k] = nullptr;
    a->czr[k] = nullptr;
    a->cchild[k] = nullptr;
    a->cshift[k] = 0;
  }
  a->ncoarse = 0;
  if (a->tmem != nullptr) dfree(A, a->has_alloc, a->tmem, a->stream);
  a->tmem = nullptr;
  a->tree = libcga::TreeView{};
}

// The occupancy tree of `a` (errors of its bounded waits land in a's header).
int build_tree(cga* a, cudaStream_t s) {
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  const libcga::TreeLayout L = libcga::tree_layout(a->grid.bits, a->lv.cap);
  const libcga::Tuning tu = libcga::tuning_for(a->grid.bits, a->lv.cap);
  void* mem = dalloc(A, L.bytes, s);
  if (mem == nullptr) return CGA_ERR_OOM;
  void* scratch = dalloc(A, libcga::tree_scratch_bytes(L, tu.radix_bits), s);
  if (scratch == nullptr) {
    dfree(A, a->has_alloc, mem, s);
    return CGA_ERR_OOM;
  }
  const int rc = cuda_rc(libcga::run_tree_build(a->lv, L, mem, scratch, tu, &a->lv.hdr->err, s));
  dfree(A, a->has_alloc, scratch, s);
  if (rc != CGA_OK) {
    dfree(A, a->has_alloc, mem, s);
    return rc;
  }
  a->tmem = mem;
  a->tree = libcga::tree_view(L, mem);
  return CGA_OK;
}

// Coarse level k of `a`: re-key the next finer level (the CGA itself for
// k = 0) by cells of 2^(shift - finer shift) of its voxels, then index each
// coarse slab's first finer slab and build the level's x directory.
int build_coarse_level(cga* a, int k, uint32_t shift, cudaStream_t s) {
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  const Levels& fine = k == 0 ? a->lv : a->clv[k - 1];
  const uint32_t dsh = shift - (k == 0 ? 0u : a->cshift[k - 1]);
  const uint32_t bc = a->grid.bits - shift;
  const uint64_t cap = std::min<uint64_t>(fine.cap, pow2(3 * bc));
  const uint64_t cap1 = std::min<uint64_t>(cap, pow2(2 * bc));
  const uint64_t cap2 = std::min<uint64_t>(cap, pow2(bc));
  const size_t lb = levels_bytes(cap, cap1, cap2, 3);
  const size_t xsb = align_up((cap2 + 1) * 4);
  const size_t xdb = align_up(((size_t)pow2(bc) + 1) * 4);
  const size_t zrb = align_up(cap1 * sizeof(uint4));
  // child-column table: skipped (searched instead) when it would be large
  const size_t chb = (cap1 << dsh) * 4 <= kChildTableMaxBytes ? align_up((cap1 << dsh) * 4) : 0;
  void* mem = dalloc(A, lb + xsb + xdb + zrb + chb, s);
  if (mem == nullptr) return CGA_ERR_OOM;
  const Levels clv = levels_carve(mem, bc, cap, cap1, cap2, 3);
  uint32_t* xs = reinterpret_cast<uint32_t*>(static_cast<char*>(mem) + lb);
  uint32_t* cxdir = reinterpret_cast<uint32_t*>(static_cast<char*>(mem) + lb + xsb);
  uint4* czr = reinterpret_cast<uint4*>(static_cast<char*>(mem) + lb + xsb + xdb);
  uint32_t* cchild =
      chb ? reinterpret_cast<uint32_t*>(static_cast<char*>(mem) + lb + xsb + xdb + zrb) : nullptr;
  libcga::SortSeg seg{};
  seg.src = fine;
  seg.plane = 3;
  seg.shift = dsh;
  seg.from_cga = 1;
  seg.bits = bc;
  seg.key_bits = 3 * bc;
  const libcga::Tuning tu = libcga::tuning_for(bc, fine.cap);
  seg.passes = libcga::radix_passes(seg.key_bits, tu.radix_bits);
  seg.num_tiles = (uint32_t)((fine.cap + libcga::kTile - 1) / libcga::kTile);
  seg.out = clv;
  const bool key64 = seg.key_bits > 32;
  const uint32_t tiles = seg.num_tiles;
  const uint64_t keys = (uint64_t)tiles * libcga::kTile;
  void* scratch = dalloc(A, libcga::sort_scratch_bytes(keys, tiles, 1, key64, tu.radix_bits), s);
  int rc = CGA_ERR_OOM;
  if (scratch != nullptr) {
    const libcga::SortScratch sc =
        libcga::sort_scratch_carve(scratch, keys, tiles, 1, key64, tu);
    cudaError_t e = libcga::run_sort_pipeline(&seg, 1, tiles, seg.passes, key64, sc, s);
    if (e == cudaSuccess) e = libcga::run_coarse_slab_index(fine, clv, dsh, xs, s);
    if (e == cudaSuccess) e = libcga::run_x_directory(clv, cxdir, s);
    if (e == cudaSuccess) e = libcga::run_column_table(clv, czr, s);
    if (e == cudaSuccess && cchild != nullptr) {
      e = libcga::run_child_columns(fine, clv, xs, dsh, cchild, s);
    }
    rc = cuda_rc(e);
    dfree(A, a->has_alloc, scratch, s);
  }
  if (rc != CGA_OK) {
    dfree(A, a->has_alloc, mem, s);
    return rc;
  }
  a->cmem[k] = mem;
  a->clv[k] = clv;
  a->xs[k] = xs;
  a->cshift[k] = shift;
  a->cxdir[k] = cxdir;
  a->czr[k] = czr;
  a->cchild[k] = cchild;
  a->ncoarse = (uint32_t)k + 1;
  return CGA_OK;
}

}  // namespace

int cga_nn_prepare_levels(cga_t* a, const uint32_t* shifts, uint32_t count, void* stream) {
  if (a == nullptr || a->view || count > CGA_NN_MAX_LEVELS || (count > 0 && shifts == nullptr)) {
    return CGA_ERR_INVALID_ARG;
  }
  const bool tree = count == 1 && shifts[0] == CGA_NN_TREE;
  for (uint32_t k = 0; k < count && !tree; ++k) {
    if (shifts[k] < 1 || shifts[k] >= a->grid.bits || shifts[k] > CGA_NN_MAX_SHIFT ||
        (k > 0 && shifts[k] <= shifts[k - 1])) {
      return CGA_ERR_INVALID_ARG;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  drop_coarse(a);
  if (a->xdmem == nullptr) {
    void* xm = dalloc(A, ((size_t)pow2(a->grid.bits) + 1) * 4, s);
    if (xm == nullptr) return CGA_ERR_OOM;
    const int rc = cuda_rc(libcga::run_x_directory(a->lv, static_cast<uint32_t*>(xm), s));
    if (rc != CGA_OK) {
      dfree(A, a->has_alloc, xm, s);
      return rc;
    }
    a->xdmem = xm;
    a->xdir = static_cast<uint32_t*>(xm);
  }
  if (a->zrmem == nullptr) {
    void* zm = dalloc(A, (size_t)std::max<uint64_t>(a->lv.cap1, 1) * sizeof(uint4), s);
    if (zm == nullptr) return CGA_ERR_OOM;
    const int rc = cuda_rc(libcga::run_column_table(a->lv, static_cast<uint4*>(zm), s));
    if (rc != CGA_OK) {
      dfree(A, a->has_alloc, zm, s);
      return rc;
    }
    a->zrmem = zm;
    a->ctab = static_cast<uint4*>(zm);
  }
  if (tree) {
    const int rc = build_tree(a, s);
    if (rc != CGA_OK) drop_coarse(a);
    return rc;
  }
  for (uint32_t k = 0; k < count; ++k) {
    const int rc = build_coarse_level(a, (int)k, shifts[k], s);
    if (rc != CGA_OK) {
      drop_coarse(a);
      return rc;
    }
  }
  return CGA_OK;
}

int cga_nn_prepare(cga_t* a, uint32_t shift, void* stream) {
  return cga_nn_prepare_levels(a, &shift, shift == 0 ? 0u : 1u, stream);
}

int cga_nn_autotune_for(cga_t* a, const float* d_q, uint64_t m, uint64_t m_per_prepare,
                        uint32_t* chosen_shifts, float* times_ms, void* stream) {
  if (a == nullptr || a->view || chosen_shifts == nullptr || m == 0 || d_q == nullptr ||
      m > libcga::kNnMaxQueries) {
    return CGA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* out = dalloc(A, (size_t)m * 12 + 256, s);
  if (out == nullptr) return CGA_ERR_OOM;
  uint32_t* idx = static_cast<uint32_t*>(out);
  uint64_t* d2 = reinterpret_cast<uint64_t*>(static_cast<char*>(out) + align_up((size_t)m * 4));
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int rc = CGA_OK;
  for (int i = 0; i < 4 && rc == CGA_OK; ++i) rc = cuda_rc(cudaEventCreate(&ev[i]));
  // candidates (coarse shifts, 0 = unused): the fine search alone, one coarse
  // level of 4..32 voxel cells, two coarse levels, the occupancy tree
  static const uint32_t cand[CGA_NN_AUTOTUNE_CANDIDATES][CGA_NN_MAX_LEVELS] = {
      {0, 0}, {2, 0}, {3, 0}, {4, 0}, {5, 0}, {2, 5}, {3, 6}, {3, 7}, {4, 8}, {CGA_NN_TREE, 0}};
  float best_ms = 0.0f;
  int best = 0;
  bool have = false;
  for (int k = 0; k < CGA_NN_AUTOTUNE_CANDIDATES && rc == CGA_OK; ++k) {
    const uint32_t count = cand[k][0] == 0 ? 0u : (cand[k][1] == 0 ? 1u : 2u);
    if (count > 0 && cand[k][0] != CGA_NN_TREE && cand[k][count - 1] >= a->grid.bits) {
      if (times_ms) times_ms[k] = -1.0f;
      continue;
    }
    rc = cuda_rc(cudaEventRecord(ev[0], s));
    if (rc == CGA_OK) rc = cga_nn_prepare_levels(a, cand[k], count, stream);
    if (rc == CGA_OK) rc = cuda_rc(cudaEventRecord(ev[1], s));
    if (rc == CGA_OK) rc = cga_nn_query(a, d_q, m, idx, d2, stream);  // warm-up
    if (rc == CGA_OK) rc = cuda_rc(cudaEventRecord(ev[2], s));
    if (rc == CGA_OK) rc = cga_nn_query(a, d_q, m, idx, d2, stream);
    if (rc == CGA_OK) rc = cuda_rc(cudaEventRecord(ev[3], s));
    if (rc == CGA_OK) rc = cuda_rc(cudaEventSynchronize(ev[3]));
    float prep = 0.0f, ms = 0.0f;
    if (rc == CGA_OK) rc = cuda_rc(cudaEventElapsedTime(&prep, ev[0], ev[1]));
    if (rc == CGA_OK) rc = cuda_rc(cudaEventElapsedTime(&ms, ev[2], ev[3]));
    if (rc != CGA_OK) break;
    // the cost per preparation: its own time and the search of the queries
    // it serves (the sample's time scaled), or the sample's search alone
    const float cost =
        m_per_prepare > 0 ? prep + ms * (float)((double)m_per_prepare / (double)m) : ms;
    if (times_ms) times_ms[k] = cost;
    if (!have || cost < best_ms) {
      best_ms = cost;
      best = k;
      have = true;
    }
  }
  const uint32_t best_count = cand[best][0] == 0 ? 0u : (cand[best][1] == 0 ? 1u : 2u);
  if (rc == CGA_OK) rc = cga_nn_prepare_levels(a, cand[best], best_count, stream);
  for (int i = 0; i < 4; ++i) {
    if (ev[i]) cudaEventDestroy(ev[i]);
  }
  dfree(A, a->has_alloc, out, s);
  if (rc == CGA_OK) {
    for (int k = 0; k < CGA_NN_MAX_LEVELS; ++k) chosen_shifts[k] = cand[best][k];
  }
  return rc;
}

int cga_nn_autotune(cga_t* a, const float* d_q, uint64_t m, uint32_t* chosen_shifts,
                    float* times_ms, void* stream) {
  return cga_nn_autotune_for(a, d_q, m, 0, chosen_shifts, times_ms, stream);
}

int cga_nn_sort_queries(const cga_t* a, const float* d_q, uint64_t m, uint64_t* d_order,
                        void* stream) {
  if (a == nullptr || (m > 0 && (d_q == nullptr || d_order == nullptr))) return CGA_ERR_INVALID_ARG;
  if (m > libcga::kNnMaxQueries) return CGA_ERR_INVALID_ARG;
  if (m == 0) return CGA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const libcga::NnSeg seg = nn_segment(a, d_q, m, nullptr, nullptr);
  const cga_allocator* A = a->has_alloc ? &a->alloc : nullptr;
  void* scratch = dalloc(A, libcga::nn_scratch_bytes(seg.num_tiles, 1), s);
  if (scratch == nullptr) return CGA_ERR_OOM;
  const libcga::NnTables t = libcga::nn_tables(scratch, seg.num_tiles, 1);
  cudaError_t e = libcga::nn_upload_one(seg, t, s);
  if (e == cudaSuccess) e = libcga::run_nn_sort_device(1, seg.num_tiles, t, s);
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(d_order, t.sort.keys0, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
  }
  dfree(A, a->has_alloc, scratch, s);
  return cuda_rc(e);
}

int cga_nn_query_ordered(const cga_t* a, const float* d_q, uint64_t m, const uint64_t* d_order,
                         uint32_t* d_idx, uint64_t* d_dist2, void* stream) {
  if (a == nullptr || (m > 0 && (d_q == nullptr || d_idx == nullptr || d_dist2 == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  if (m > libcga::kNnMaxQueries) return CGA_ERR_INVALID_ARG;
  const libcga::NnSeg seg = nn_segment(a, d_q, m, d_idx, d_dist2);
  return cuda_rc(libcga::run_nn_search(seg, reinterpret_cast<const unsigned long long*>(d_order),
                                       static_cast<cudaStream_t>(stream)));
}

int cga_decode(const cga_t* a, uint32_t* d_xyz, void* stream) {
  if (a == nullptr || (d_xyz == nullptr && a->lv.cap > 0)) return CGA_ERR_INVALID_ARG;
  return cuda_rc(libcga::run_decode(a->lv, d_xyz, static_cast<cudaStream_t>(stream)));
}

int cga_info(const cga_t* a, cga_sizes* out) {
  if (a == nullptr || out == nullptr) return CGA_ERR_INVALID_ARG;
  Header hd{};
  const int rc = read_header(a->lv, a->stream, &hd);
  if (rc != CGA_OK) return rc;
  out->u = hd.cnt[0];
  out->g = hd.cnt[1];
  out->h = hd.cnt[2];
  out->bytes = 2 * out->h + 4 * (out->h + 1) + 2 * out->g + 4 * (out->g + 1) + 2 * out->u;
  out->capacity = a->lv.cap;
  return err_from_bits(hd.err);
}

int cga_view(const cga_t* a, cga_arrays* out) {
  if (a == nullptr || out == nullptr) return CGA_ERR_INVALID_ARG;
  cga_sizes sz{};
  const int rc = cga_info(a, &sz);
  out->grid = a->grid;
  out->h = sz.h;
  out->g = sz.g;
  out->u = sz.u;
  out->X_index = a->lv.idx2;
  out->X_pointer = a->lv.ptr2;
  out->Y_index = a->lv.idx1;
  out->Y_pointer = a->lv.ptr1;
  out->Z_index = a->lv.idx0;
  return rc;
}

int cga2d_info(const cga2d_t* p, uint64_t* h, uint64_t* g) {
  if (p == nullptr || h == nullptr || g == nullptr) return CGA_ERR_INVALID_ARG;
  Header hd{};
  const int rc = read_header(p->lv, p->stream, &hd);
  if (rc != CGA_OK) return rc;
  *g = hd.cnt[0];
  *h = hd.cnt[1];
  return err_from_bits(hd.err);
}

int cga2d_view(const cga2d_t* p, cga2d_arrays* out) {
  if (p == nullptr || out == nullptr) return CGA_ERR_INVALID_ARG;
  uint64_t h = 0, g = 0;
  const int rc = cga2d_info(p, &h, &g);
  out->bits = p->bits;
  out->plane = p->plane;
  out->h = h;
  out->g = g;
  out->U_index = p->lv.idx1;
  out->U_pointer = p->lv.ptr1;
  out->V_index = p->lv.idx0;
  return rc;
}

int cga_download(const cga_t* a, uint16_t* h_X_index, uint32_t* h_X_pointer,
                 uint16_t* h_Y_index, uint32_t* h_Y_pointer, uint16_t* h_Z_index) {
  if (a == nullptr || h_X_pointer == nullptr || h_Y_pointer == nullptr) {
    return CGA_ERR_INVALID_ARG;
  }
  cga_sizes sz{};
  int rc = cga_info(a, &sz);
  if (rc != CGA_OK && rc != CGA_ERR_NONFINITE && rc != CGA_ERR_TIMEOUT &&
      rc != CGA_ERR_INTERNAL) {
    return rc;
  }
  if ((sz.h && !h_X_index) || (sz.g && !h_Y_index) || (sz.u && !h_Z_index)) {
    return CGA_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaSuccess;
  if (sz.h) e = cudaMemcpy(h_X_index, a->lv.idx2, sz.h * 2, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_X_pointer, a->lv.ptr2, (sz.h + 1) * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && sz.g) e = cudaMemcpy(h_Y_index, a->lv.idx1, sz.g * 2, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_Y_pointer, a->lv.ptr1, (sz.g + 1) * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && sz.u) e = cudaMemcpy(h_Z_index, a->lv.idx0, sz.u * 2, cudaMemcpyDeviceToHost);
  const int rc2 = cuda_rc(e);
  return rc2 != CGA_OK ? rc2 : rc;
}

int cga2d_download(const cga2d_t* p, uint16_t* h_U_index, uint32_t* h_U_pointer,
                   uint16_t* h_V_index) {
  if (p == nullptr || h_U_pointer == nullptr) return CGA_ERR_INVALID_ARG;
  uint64_t h = 0, g = 0;
  int rc = cga2d_info(p, &h, &g);
  if (rc == CGA_ERR_CUDA || rc == CGA_ERR_INVALID_ARG) return rc;
  if ((h && !h_U_index) || (g && !h_V_index)) return CGA_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (h) e = cudaMemcpy(h_U_index, p->lv.idx1, h * 2, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_U_pointer, p->lv.ptr1, (h + 1) * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && g) e = cudaMemcpy(h_V_index, p->lv.idx0, g * 2, cudaMemcpyDeviceToHost);
  const int rc2 = cuda_rc(e);
  return rc2 != CGA_OK ? rc2 : rc;
}

void cga_free(cga_t* a) { release(a); }

void cga2d_free(cga2d_t* p) {
  if (p == nullptr || p->view) return;
  dfree(&p->alloc, p->has_alloc, p->mem, p->stream);
  delete p;
}


// ------------------------------------------------------------------ batches

int cga_build_batch(const cga_cloud* clouds, uint32_t count, const cga_allocator* A,
                    void* stream, cga_t** out) {
  if (out == nullptr || (count > 0 && clouds == nullptr)) return CGA_ERR_INVALID_ARG;
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < count; ++i) {
    const cga_cloud& c = clouds[i];
    if (!grid_ok(&c.grid) || c.n > CGA_MAX_POINTS || (c.n > 0 && c.d_xyz == nullptr)) {
      return CGA_ERR_INVALID_ARG;
    }
  }
  if (count == 0) return CGA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t max_bits = 1;
  uint64_t max_n = 0;
  for (uint32_t i = 0; i < count; ++i) {
    max_bits = std::max(max_bits, clouds[i].grid.bits);
    max_n = std::max<uint64_t>(max_n, clouds[i].n);
  }
  const libcga::Tuning tu = libcga::tuning_for(max_bits, max_n);
  std::vector<libcga::SortSeg> segs(count);
  std::vector<cga*> hs(count, nullptr);
  uint64_t tiles = 0;
  uint32_t max_passes = 0;
  bool key64 = false;
  int rc = CGA_OK;
  for (uint32_t i = 0; i < count && rc == CGA_OK; ++i) {
    const cga_cloud& c = clouds[i];
    hs[i] = new_cga(c.grid, A, s, c.n);
    if (hs[i] == nullptr) {
      rc = CGA_ERR_OOM;
      break;
    }
    libcga::SortSeg& sg = segs[i];
    sg = libcga::SortSeg{};
    sg.xyz = c.d_xyz;
    sg.scale = c.grid.scale;
    for (int a = 0; a < 3; ++a) sg.off[a] = c.grid.offset[a];
    if (c.h_xform12 != nullptr) {
      std::memcpy(sg.X, c.h_xform12, sizeof(sg.X));
      sg.has_x = 1;
    }
    sg.n_host = (uint32_t)c.n;
    sg.bits = c.grid.bits;
    sg.key_bits = 3 * c.grid.bits;
    sg.passes = libcga::radix_passes(sg.key_bits, tu.radix_bits);
    sg.tile_base = (uint32_t)tiles;
    sg.num_tiles = (uint32_t)((c.n + libcga::kTile - 1) / libcga::kTile);
    sg.key_base = tiles * libcga::kTile;
    sg.out = hs[i]->lv;
    tiles += sg.num_tiles;
    max_passes = std::max(max_passes, sg.passes);
    key64 = key64 || sg.key_bits > 32;
  }
  if (rc == CGA_OK && tiles > 0xFFFFFFFFull / libcga::kTile) rc = CGA_ERR_INVALID_ARG;
  void* scratch = nullptr;
  if (rc == CGA_OK) {
    const uint64_t keys = tiles * libcga::kTile;
    scratch = dalloc(
        A, libcga::sort_scratch_bytes(keys, (uint32_t)tiles, (int)count, key64, tu.radix_bits), s);
    if (scratch == nullptr) rc = CGA_ERR_OOM;
    if (rc == CGA_OK) {
      const libcga::SortScratch sc =
          libcga::sort_scratch_carve(scratch, keys, (uint32_t)tiles, (int)count, key64, tu);
      rc = cuda_rc(libcga::run_sort_pipeline(segs.data(), (int)count, (uint32_t)tiles,
                                             max_passes, key64, sc, s));
      dfree(A, A != nullptr, scratch, s);
    }
  }
  if (rc != CGA_OK) {
    for (cga* h : hs) release(h);
    return rc;
  }
  for (uint32_t i = 0; i < count; ++i) out[i] = hs[i];
  return CGA_OK;
}

namespace {

// Merge pair table + output handles for `count` pairs.
int plan_merges(const cga_t* const* a, const cga_t* const* b, uint32_t count,
                const cga_allocator* A, cudaStream_t s, std::vector<libcga::MergePair>& pairs,
                std::vector<cga*>& hs, uint32_t& total_spl, uint32_t& total_tiles,
                uint32_t& half) {
  pairs.assign(count, libcga::MergePair{});
  hs.assign(count, nullptr);
  uint64_t spl = 0, tiles = 0;
  uint32_t max_bits = 1;
  uint64_t max_in = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (a[i] == nullptr || b[i] == nullptr) return CGA_ERR_INVALID_ARG;
    if (!same_grid(a[i]->grid, b[i]->grid)) return CGA_ERR_GRID_MISMATCH;
    const uint64_t cap = std::min<uint64_t>(a[i]->lv.cap + b[i]->lv.cap, pow2(3 * a[i]->grid.bits));
    if (cap > CGA_MAX_POINTS) return CGA_ERR_INVALID_ARG;
    max_bits = std::max(max_bits, a[i]->grid.bits);
    max_in = std::max<uint64_t>(max_in, a[i]->lv.cap + b[i]->lv.cap);
  }
  half = libcga::tuning_for(max_bits, max_in).merge_half;
  for (uint32_t i = 0; i < count; ++i) {
    const uint64_t cap = std::min<uint64_t>(a[i]->lv.cap + b[i]->lv.cap, pow2(3 * a[i]->grid.bits));
    hs[i] = new_cga(a[i]->grid, A, s, cap);
    if (hs[i] == nullptr) return CGA_ERR_OOM;
    libcga::MergePair& P = pairs[i];
    P.a = a[i]->lv;
    P.b = b[i]->lv;
    P.out = hs[i]->lv;
    P.spl_a = libcga::merge_splitters(a[i]->lv.cap, half);
    P.spl_b = libcga::merge_splitters(b[i]->lv.cap, half);
    P.spl_base = (uint32_t)spl;
    P.tile_base = (uint32_t)tiles;
    P.num_tiles = P.spl_a + P.spl_b + 1;
    spl += P.spl_a + P.spl_b;
    tiles += P.num_tiles;
    if (tiles > 0x7FFFFFFFull) return CGA_ERR_INVALID_ARG;
  }
  total_spl = (uint32_t)spl;
  total_tiles = (uint32_t)tiles;
  return CGA_OK;
}

}  // namespace

int cga_merge_batch(const cga_t* const* a, const cga_t* const* b, uint32_t count,
                    const cga_allocator* A, void* stream, cga_t** out) {
  if (out == nullptr || (count > 0 && (a == nullptr || b == nullptr))) return CGA_ERR_INVALID_ARG;
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  if (count == 0) return CGA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<libcga::MergePair> pairs;
  std::vector<cga*> hs;
  uint32_t total_spl = 0, total_tiles = 0, half = libcga::kMergeHalf;
  int rc = plan_merges(a, b, count, A, s, pairs, hs, total_spl, total_tiles, half);
  if (rc == CGA_OK) {
    void* scratch = dalloc(A, libcga::merge_scratch_bytes(total_spl, total_tiles, (int)count), s);
    if (scratch == nullptr) {
      rc = CGA_ERR_OOM;
    } else {
      const libcga::MergeScratch sc =
          libcga::merge_scratch_carve(scratch, total_spl, total_tiles, (int)count, half);
      rc = cuda_rc(libcga::run_merge(pairs.data(), (int)count, total_spl, total_tiles, sc, s));
      dfree(A, A != nullptr, scratch, s);
    }
  }
  if (rc != CGA_OK) {
    for (cga* h : hs) release(h);
    return rc;
  }
  for (uint32_t i = 0; i < count; ++i) out[i] = hs[i];
  return CGA_OK;
}

int cga_project_batch(const cga_t* const* a, const int* planes, uint32_t count,
                      const cga_allocator* A, void* stream, cga2d_t** out) {
  if (out == nullptr || (count > 0 && (a == nullptr || planes == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < count; ++i) {
    if (a[i] == nullptr || planes[i] < CGA_PLANE_XY || planes[i] > CGA_PLANE_YZ) {
      return CGA_ERR_INVALID_ARG;
    }
  }
  if (count == 0) return CGA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<cga2d*> ps(count, nullptr);
  std::vector<libcga::ProjPair> xy;
  std::vector<libcga::SortSeg> segs;
  std::vector<uint32_t> bitmap;  // xz / yz projections of small grids (no sort)
  uint64_t tiles = 0, max_cap1 = 0;
  int rc = CGA_OK;
  for (uint32_t i = 0; i < count && rc == CGA_OK; ++i) {
    const uint32_t b = a[i]->grid.bits;
    uint64_t cap, cap1;
    if (planes[i] == CGA_PLANE_XY) {
      cap = a[i]->lv.cap1;
      cap1 = a[i]->lv.cap2;
    } else {
      cap = std::min<uint64_t>(a[i]->lv.cap, pow2(2 * b));
      cap1 = std::min<uint64_t>(cap, pow2(b));
    }
    void* mem = dalloc(A, levels_bytes(cap, cap1, 0, 2), s);
    cga2d* p = mem ? new (std::nothrow) cga2d{} : nullptr;
    if (p == nullptr) {
      if (mem) dfree(A, A != nullptr, mem, s);
      rc = CGA_ERR_OOM;
      break;
    }
    p->bits = b;
    p->plane = planes[i];
    p->lv = levels_carve(mem, b, cap, cap1, 0, 2);
    p->mem = mem;
    p->has_alloc = A != nullptr;
    if (A != nullptr) p->alloc = *A;
    p->stream = s;
    ps[i] = p;
    if (planes[i] == CGA_PLANE_XY) {
      xy.push_back(libcga::ProjPair{a[i]->lv, p->lv});
      max_cap1 = std::max<uint64_t>(max_cap1, a[i]->lv.cap1);
    } else if (b >= libcga::kProjBitmapMinBits && b <= libcga::kProjBitmapMaxBits) {
      bitmap.push_back(i);
    } else {
      libcga::SortSeg sg{};
      sg.src = a[i]->lv;
      sg.plane = planes[i];
      sg.from_cga = 1;
      sg.bits = b;
      sg.key_bits = 2 * b;
      sg.tile_base = (uint32_t)tiles;
      sg.num_tiles = (uint32_t)((a[i]->lv.cap + libcga::kTile - 1) / libcga::kTile);
      sg.key_base = tiles * libcga::kTile;
      sg.out = p->lv;
      tiles += sg.num_tiles;
      segs.push_back(sg);
    }
  }
  if (rc == CGA_OK && !xy.empty()) {
    void* tab = dalloc(A, sizeof(libcga::ProjPair) * xy.size(), s);
    if (tab == nullptr) {
      rc = CGA_ERR_OOM;
    } else {
      cudaError_t e = cudaMemcpyAsync(tab, xy.data(), sizeof(libcga::ProjPair) * xy.size(),
                                      cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) {
        e = libcga::run_project_xy_device(static_cast<libcga::ProjPair*>(tab), (int)xy.size(),
                                          max_cap1, s);
      }
      rc = cuda_rc(e);
      dfree(A, A != nullptr, tab, s);
    }
  }
  if (rc == CGA_OK && !bitmap.empty()) {
    uint32_t max_bits = 0;
    for (uint32_t i : bitmap) max_bits = std::max(max_bits, a[i]->grid.bits);
    void* scratch = dalloc(A, libcga::project_bitmap_scratch_bytes(max_bits), s);
    if (scratch == nullptr) {
      rc = CGA_ERR_OOM;
    } else {
      for (uint32_t i : bitmap) {
        if (rc != CGA_OK) break;
        rc = cuda_rc(libcga::run_project_bitmap(a[i]->lv, planes[i], ps[i]->lv, scratch, s));
      }
      dfree(A, A != nullptr, scratch, s);
    }
  }
  if (rc == CGA_OK && !segs.empty()) {
    uint32_t max_bits = 1;
    uint64_t max_cap = 0;
    for (const auto& sg : segs) {
      max_bits = std::max(max_bits, sg.bits);
      max_cap = std::max<uint64_t>(max_cap, sg.src.cap);
    }
    const libcga::Tuning tu = libcga::tuning_for(max_bits, max_cap);
    uint32_t max_passes = 0;
    for (auto& sg : segs) {
      sg.passes = libcga::radix_passes(sg.key_bits, tu.radix_bits);
      max_passes = std::max(max_passes, sg.passes);
    }
    const uint64_t keys = tiles * libcga::kTile;
    void* scratch = dalloc(
        A, libcga::sort_scratch_bytes(keys, (uint32_t)tiles, (int)segs.size(), false, tu.radix_bits),
        s);
    if (scratch == nullptr) {
      rc = CGA_ERR_OOM;
    } else {
      const libcga::SortScratch sc =
          libcga::sort_scratch_carve(scratch, keys, (uint32_t)tiles, (int)segs.size(), false, tu);
      rc = cuda_rc(libcga::run_sort_pipeline(segs.data(), (int)segs.size(), (uint32_t)tiles,
                                             max_passes, false, sc, s));
      dfree(A, A != nullptr, scratch, s);
    }
  }
  if (rc != CGA_OK) {
    for (cga2d* p : ps) cga2d_free(p);
    return rc;
  }
  for (uint32_t i = 0; i < count; ++i) out[i] = ps[i];
  return CGA_OK;
}

int cga_nn_query_batch(const cga_t* const* a, const cga_queries* q, uint32_t count,
                       const cga_allocator* A, void* stream) {
  if (count > 0 && (a == nullptr || q == nullptr)) return CGA_ERR_INVALID_ARG;
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  std::vector<libcga::NnSeg> segs;
  uint64_t tiles = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (a[i] == nullptr || q[i].m > libcga::kNnMaxQueries) return CGA_ERR_INVALID_ARG;
    if (q[i].m > 0 && (q[i].d_q == nullptr || q[i].d_idx == nullptr || q[i].d_dist2 == nullptr)) {
      return CGA_ERR_INVALID_ARG;
    }
    if (q[i].m == 0) continue;
    libcga::NnSeg sg{};
    sg.a = a[i]->lv;
    sg.scale = a[i]->grid.scale;
    for (int k = 0; k < 3; ++k) sg.off[k] = a[i]->grid.offset[k];
    sg.q = q[i].d_q;
    sg.m = (uint32_t)q[i].m;
    sg.idx = q[i].d_idx;
    sg.d2 = reinterpret_cast<unsigned long long*>(q[i].d_dist2);
    sg.tile_base = (uint32_t)tiles;
    sg.num_tiles = (uint32_t)((q[i].m + libcga::kTile - 1) / libcga::kTile);
    attach_coarse(a[i], sg);
    tiles += sg.num_tiles;
    segs.push_back(sg);
  }
  if (segs.empty()) return CGA_OK;
  if (tiles > 0xFFFFFFFFull / libcga::kTile) return CGA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = dalloc(A, libcga::nn_scratch_bytes((uint32_t)tiles, (int)segs.size()), s);
  if (scratch == nullptr) return CGA_ERR_OOM;
  const int rc = cuda_rc(libcga::run_nn(segs.data(), (int)segs.size(), (uint32_t)tiles, scratch, s));
  dfree(A, A != nullptr, scratch, s);
  return rc;
}

// ----------------------------------------------------------------- pipeline

struct cga_pipeline {
  uint32_t S = 0;
  std::vector<cga> views;      // 3 per item: cloud, twin, merged
  std::vector<cga2d> xy;       // 1 per item
  void* arena = nullptr;
  cga_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t stream = nullptr;
  libcga::SortScratch build{};
  uint32_t build_tiles = 0, build_passes = 0;
  bool key64 = false;
  libcga::MergeScratch merge{};
  uint32_t merge_spl = 0, merge_tiles = 0;
  libcga::ProjPair* d_proj = nullptr;
  uint64_t max_cap1 = 0;
  libcga::NnTables nn{};
  uint32_t nn_tiles = 0, nn_segs = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t graph_kernels = 0;
};

namespace {

struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += align_up(bytes);
    return o;
  }
};

int pipeline_queue(cga_pipeline* p, cudaStream_t s) {
  cudaError_t e = libcga::run_sort_device((int)(2 * p->S), p->build_tiles, p->build_passes,
                                          p->key64, 3, p->build, s);
  if (e == cudaSuccess) e = libcga::run_merge_device((int)p->S, p->merge_spl, p->merge_tiles, p->merge, s);
  if (e == cudaSuccess) e = libcga::run_project_xy_device(p->d_proj, (int)p->S, p->max_cap1, s);
  if (e == cudaSuccess && p->nn_segs > 0) {
    e = libcga::run_nn_device((int)p->nn_segs, p->nn_tiles, p->nn, s);
  }
  return cuda_rc(e);
}

}  // namespace

int cga_pipeline_create(const cga_pipeline_item* items, uint32_t count, const cga_allocator* A,
                        void* stream, cga_pipeline_t** out) {
  if (out == nullptr || count == 0 || items == nullptr) return CGA_ERR_INVALID_ARG;
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < count; ++i) {
    const cga_pipeline_item& it = items[i];
    if (!grid_ok(&it.grid) || it.n > CGA_MAX_POINTS / 2 || (it.n > 0 && it.d_xyz == nullptr) ||
        it.m > libcga::kNnMaxQueries ||
        (it.m > 0 && (it.d_q == nullptr || it.d_idx == nullptr || it.d_dist2 == nullptr))) {
      return CGA_ERR_INVALID_ARG;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cga_pipeline* p = new (std::nothrow) cga_pipeline();
  if (p == nullptr) return CGA_ERR_OOM;
  const uint32_t S = count;
  p->S = S;
  p->stream = s;
  p->has_alloc = A != nullptr;
  if (A != nullptr) p->alloc = *A;
  // --- launch shapes: one per pipeline, from its largest item
  uint32_t max_bits = 1;
  uint64_t max_n = 0;
  for (uint32_t i = 0; i < S; ++i) {
    max_bits = std::max(max_bits, items[i].grid.bits);
    max_n = std::max<uint64_t>(max_n, items[i].n);
  }
  const libcga::Tuning tu = libcga::tuning_for(max_bits, max_n);
  const uint32_t half = tu.merge_half;
  // --- layout
  Bump bump;
  std::vector<size_t> lv_off(4 * (size_t)S);
  std::vector<uint64_t> caps(3 * (size_t)S);
  uint64_t build_tiles = 0, spl = 0, mtiles = 0, nn_tiles = 0;
  uint32_t nn_segs = 0;
  for (uint32_t i = 0; i < S; ++i) {
    const uint32_t b = items[i].grid.bits;
    const uint64_t n = items[i].n;
    const uint64_t cm = std::min<uint64_t>(2 * n, pow2(3 * b));
    caps[3 * i] = n;
    caps[3 * i + 1] = n;
    caps[3 * i + 2] = cm;
    for (int k = 0; k < 3; ++k) {
      const uint64_t c = caps[3 * i + k];
      lv_off[4 * i + k] =
          bump.take(levels_bytes(c, std::min<uint64_t>(c, pow2(2 * b)), std::min<uint64_t>(c, pow2(b)), 3));
    }
    const uint64_t pc = std::min<uint64_t>(cm, pow2(2 * b)), pc1 = std::min<uint64_t>(cm, pow2(b));
    lv_off[4 * i + 3] = bump.take(levels_bytes(pc, pc1, 0, 2));
    const uint64_t t = (n + libcga::kTile - 1) / libcga::kTile;
    build_tiles += 2 * t;
    const uint64_t sa = libcga::merge_splitters(n, half);
    spl += 2 * sa;
    mtiles += 2 * sa + 1;
    if (items[i].m > 0) {
      nn_tiles += (items[i].m + libcga::kTile - 1) / libcga::kTile;
      ++nn_segs;
    }
  }
  if (build_tiles > 0xFFFFFFFFull / libcga::kTile || nn_tiles > 0xFFFFFFFFull / libcga::kTile ||
      mtiles > 0x7FFFFFFFull) {
    delete p;
    return CGA_ERR_INVALID_ARG;
  }
  bool key64 = false;
  uint32_t passes = 0;
  for (uint32_t i = 0; i < S; ++i) {
    key64 = key64 || 3 * items[i].grid.bits > 32;
    passes = std::max<uint32_t>(passes, libcga::radix_passes(3 * items[i].grid.bits, tu.radix_bits));
  }
  const size_t o_build = bump.take(libcga::sort_scratch_bytes(
      build_tiles * libcga::kTile, (uint32_t)build_tiles, (int)(2 * S), key64, tu.radix_bits));
  const size_t o_merge = bump.take(libcga::merge_scratch_bytes((uint32_t)spl, (uint32_t)mtiles, (int)S));
  const size_t o_proj = bump.take(sizeof(libcga::ProjPair) * S);
  const size_t o_nn = bump.take(nn_segs ? libcga::nn_scratch_bytes((uint32_t)nn_tiles, (int)nn_segs) : 0);
  p->arena = dalloc(A, bump.off, s);
  if (p->arena == nullptr) {
    delete p;
    return CGA_ERR_OOM;
  }
  char* base = static_cast<char*>(p->arena);
  // --- views
  p->views.resize(3 * (size_t)S);
  p->xy.resize(S);
  for (uint32_t i = 0; i < S; ++i) {
    const uint32_t b = items[i].grid.bits;
    for (int k = 0; k < 3; ++k) {
      const uint64_t c = caps[3 * i + k];
      cga& v = p->views[3 * i + k];
      v.grid = items[i].grid;
      v.lv = levels_carve(base + lv_off[4 * i + k], b, c, std::min<uint64_t>(c, pow2(2 * b)),
                          std::min<uint64_t>(c, pow2(b)), 3);
      v.mem = nullptr;
      v.stream = s;
      v.view = true;
    }
    const uint64_t cm = caps[3 * i + 2];
    cga2d& x = p->xy[i];
    x.bits = b;
    x.plane = CGA_PLANE_XY;
    x.lv = levels_carve(base + lv_off[4 * i + 3], b, std::min<uint64_t>(cm, pow2(2 * b)),
                        std::min<uint64_t>(cm, pow2(b)), 0, 2);
    x.mem = nullptr;
    x.stream = s;
    x.view = true;
  }
  // --- tables
  std::vector<libcga::SortSeg> bsegs(2 * (size_t)S);
  uint64_t tb = 0;
  for (uint32_t i = 0; i < S; ++i) {
    for (int k = 0; k < 2; ++k) {
      libcga::SortSeg& sg = bsegs[2 * i + k];
      sg = libcga::SortSeg{};
      sg.xyz = items[i].d_xyz;
      sg.scale = items[i].grid.scale;
      for (int a = 0; a < 3; ++a) sg.off[a] = items[i].grid.offset[a];
      if (k == 1) {
        std::memcpy(sg.X, items[i].xform12, sizeof(sg.X));
        sg.has_x = 1;
      }
      sg.n_host = (uint32_t)items[i].n;
      sg.bits = items[i].grid.bits;
      sg.key_bits = 3 * sg.bits;
      sg.passes = libcga::radix_passes(sg.key_bits, tu.radix_bits);
      sg.tile_base = (uint32_t)tb;
      sg.num_tiles = (uint32_t)((items[i].n + libcga::kTile - 1) / libcga::kTile);
      sg.key_base = tb * libcga::kTile;
      sg.out = p->views[3 * i + k].lv;
      tb += sg.num_tiles;
    }
  }
  p->build = libcga::sort_scratch_carve(base + o_build, build_tiles * libcga::kTile,
                                        (uint32_t)build_tiles, (int)(2 * S), key64, tu);
  p->build_tiles = (uint32_t)build_tiles;
  p->build_passes = passes;
  p->key64 = key64;
  std::vector<libcga::MergePair> pairs(S);
  uint64_t sb = 0, mb = 0;
  for (uint32_t i = 0; i < S; ++i) {
    libcga::MergePair& P = pairs[i];
    P.a = p->views[3 * i].lv;
    P.b = p->views[3 * i + 1].lv;
    P.out = p->views[3 * i + 2].lv;
    P.spl_a = P.spl_b = libcga::merge_splitters(items[i].n, half);
    P.spl_base = (uint32_t)sb;
    P.tile_base = (uint32_t)mb;
    P.num_tiles = P.spl_a + P.spl_b + 1;
    sb += P.spl_a + P.spl_b;
    mb += P.num_tiles;
  }
  p->merge =
      libcga::merge_scratch_carve(base + o_merge, (uint32_t)spl, (uint32_t)mtiles, (int)S, half);
  p->merge.key_level = S > 0;
  for (uint32_t i = 0; i < S; ++i) {
    p->merge.key_level = p->merge.key_level && libcga::merge_key_level(pairs[i].a.bits);
  }
  p->merge_spl = (uint32_t)spl;
  p->merge_tiles = (uint32_t)mtiles;
  std::vector<libcga::ProjPair> proj(S);
  for (uint32_t i = 0; i < S; ++i) {
    proj[i] = libcga::ProjPair{p->views[3 * i + 2].lv, p->xy[i].lv};
    p->max_cap1 = std::max<uint64_t>(p->max_cap1, p->views[3 * i + 2].lv.cap1);
  }
  p->d_proj = reinterpret_cast<libcga::ProjPair*>(base + o_proj);
  std::vector<libcga::NnSeg> nsegs;
  uint64_t nt = 0;
  for (uint32_t i = 0; i < S; ++i) {
    if (items[i].m == 0) continue;
    libcga::NnSeg sg{};
    sg.a = p->views[3 * i + 2].lv;
    sg.scale = items[i].grid.scale;
    for (int k = 0; k < 3; ++k) sg.off[k] = items[i].grid.offset[k];
    sg.q = items[i].d_q;
    sg.m = (uint32_t)items[i].m;
    sg.idx = items[i].d_idx;
    sg.d2 = reinterpret_cast<unsigned long long*>(items[i].d_dist2);
    sg.tile_base = (uint32_t)nt;
    sg.num_tiles = (uint32_t)((items[i].m + libcga::kTile - 1) / libcga::kTile);
    nt += sg.num_tiles;
    nsegs.push_back(sg);
  }
  p->nn_segs = nn_segs;
  p->nn_tiles = (uint32_t)nn_tiles;
  cudaError_t e = cudaMemcpyAsync(p->build.segs, bsegs.data(), sizeof(libcga::SortSeg) * bsegs.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(p->merge.pairs, pairs.data(), sizeof(libcga::MergePair) * S,
                        cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(p->d_proj, proj.data(), sizeof(libcga::ProjPair) * S,
                        cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess && nn_segs > 0) {
    p->nn = libcga::nn_tables(base + o_nn, (uint32_t)nn_tiles, (int)nn_segs);
    e = libcga::nn_upload(nsegs.data(), (int)nn_segs, p->nn, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dfree(A, A != nullptr, p->arena, s);
    delete p;
    return cuda_rc(e);
  }
  *out = p;
  return CGA_OK;
}

int cga_pipeline_run(cga_pipeline_t* p, void* stream) {
  if (p == nullptr) return CGA_ERR_INVALID_ARG;
  return pipeline_queue(p, static_cast<cudaStream_t>(stream));
}

int cga_pipeline_run_graph(cga_pipeline_t* p, void* stream) {
  if (p == nullptr) return CGA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->exec == nullptr) {
    cudaError_t e = cudaSuccess;
    if (p->cap_stream == nullptr) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = libcga::init_sort_kernels();  // kernel attributes before capture
    libcga::init_nn_kernels();
    if (e != cudaSuccess) return cuda_rc(e);
    const uint64_t k0 = libcga::g_launches.load();
    e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_rc(e);
    const int rc = pipeline_queue(p, p->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->cap_stream, &g);
    if (rc != CGA_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != CGA_OK ? rc : cuda_rc(e);
    }
    p->graph_kernels = libcga::g_launches.load() - k0;
    libcga::g_launches.fetch_sub(p->graph_kernels);  // counted on each replay instead
    e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      p->exec = nullptr;
      return cuda_rc(e);
    }
    p->graph = g;
  }
  libcga::count_launch((unsigned)p->graph_kernels);
  return cuda_rc(cudaGraphLaunch(p->exec, s));
}

int cga_pipeline_view(const cga_pipeline_t* p, uint32_t i, int which, const cga_t** out) {
  if (p == nullptr || out == nullptr || i >= p->S || which < 0 || which > 2) return CGA_ERR_INVALID_ARG;
  *out = &p->views[3 * (size_t)i + which];
  return CGA_OK;
}

int cga_pipeline_view_xy(const cga_pipeline_t* p, uint32_t i, const cga2d_t** out) {
  if (p == nullptr || out == nullptr || i >= p->S) return CGA_ERR_INVALID_ARG;
  *out = &p->xy[i];
  return CGA_OK;
}

void cga_pipeline_free(cga_pipeline_t* p) {
  if (p == nullptr) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap_stream) {
    cudaStreamSynchronize(p->cap_stream);
    cudaStreamDestroy(p->cap_stream);
  }
  dfree(p->has_alloc ? &p->alloc : nullptr, p->has_alloc, p->arena, p->stream);
  delete p;
}

int cga_selftest_wait_timeout(void* stream, int* observed) {
  if (observed == nullptr) return CGA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = dalloc(nullptr, libcga::wait_selftest_bytes(), s);
  if (scratch == nullptr) return CGA_ERR_OOM;
  cudaError_t e = libcga::run_wait_selftest(scratch, s);
  Header hd{};
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(&hd, scratch, sizeof(Header), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(nullptr, false, scratch, s);
  if (e != cudaSuccess) return cuda_rc(e);
  *observed = err_from_bits(hd.err);
  return CGA_OK;
}

uint64_t cga_kernel_launches(void) { return libcga::g_launches.load(std::memory_order_relaxed); }

const char* cga_strerror(int code) {
  switch (code) {
    case CGA_OK: return "ok";
    case CGA_ERR_INVALID_ARG: return "invalid argument";
    case CGA_ERR_NONFINITE: return "non-finite input point";
    case CGA_ERR_GRID_MISMATCH: return "CGAs are on different grids";
    case CGA_ERR_OOM: return "device allocation failed";
    case CGA_ERR_CUDA: return "CUDA runtime error";
    case CGA_ERR_TIMEOUT: return "bounded device wait ran out";
    case CGA_ERR_INTERNAL: return "device consistency check failed";
    case CGA_ERR_CAPACITY: return "request larger than the fixed scratch of a no-allocation call";
    default: return "unknown error";
  }
}

}  // extern "C"
