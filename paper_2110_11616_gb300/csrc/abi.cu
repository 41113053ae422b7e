// C-ABI of libcga (include/cga.h): argument checks, handle and memory
// management, and the launch sequences of the kernels in k_sort.cu / k_ops.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>

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
};

struct cga2d {
  uint32_t bits;
  int plane;
  Levels lv;
  void* mem;
  cga_allocator alloc;
  bool has_alloc;
  cudaStream_t stream;
};

namespace libcga {
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
  if (h == nullptr) return;
  dfree(&h->alloc, h->has_alloc, h->mem, h->stream);
  delete h;
}

}  // namespace

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
  seg.passes = (seg.key_bits + libcga::kRadixBits - 1) / libcga::kRadixBits;
  seg.key_base = 0;
  seg.tile_base = 0;
  seg.num_tiles = (uint32_t)((n + libcga::kTile - 1) / libcga::kTile);
  seg.out = h->lv;
  const bool key64 = seg.key_bits > 32;
  const uint32_t tiles = seg.num_tiles;
  const uint64_t keys = (uint64_t)tiles * libcga::kTile;
  void* scratch = dalloc(A, libcga::sort_scratch_bytes(keys, tiles, 1, key64), s);
  if (scratch == nullptr) {
    release(h);
    return CGA_ERR_OOM;
  }
  const libcga::SortScratch sc = libcga::sort_scratch_carve(scratch, keys, tiles, 1, key64);
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
  P.spl_a = a->lv.cap > 0 ? (uint32_t)((a->lv.cap - 1) / libcga::kMergeHalf) : 0u;
  P.spl_b = b->lv.cap > 0 ? (uint32_t)((b->lv.cap - 1) / libcga::kMergeHalf) : 0u;
  P.tile_base = 0;
  P.num_tiles = P.spl_a + P.spl_b + 1;
  const uint32_t total_spl = P.spl_a + P.spl_b;
  void* scratch = dalloc(A, libcga::merge_scratch_bytes(total_spl, P.num_tiles, 1), s);
  if (scratch == nullptr) {
    release(h);
    return CGA_ERR_OOM;
  }
  const libcga::MergeScratch sc = libcga::merge_scratch_carve(scratch, total_spl, P.num_tiles, 1);
  const int rc = cuda_rc(libcga::run_merge(&P, 1, total_spl, P.num_tiles, sc, s));
  dfree(A, A != nullptr, scratch, s);
  if (rc != CGA_OK) {
    release(h);
    return rc;
  }
  *out = h;
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
  } else {
    libcga::SortSeg seg{};
    seg.src = a->lv;
    seg.plane = plane;
    seg.from_cga = 1;
    seg.bits = b;
    seg.key_bits = 2 * b;
    seg.passes = (seg.key_bits + libcga::kRadixBits - 1) / libcga::kRadixBits;
    seg.num_tiles = (uint32_t)((a->lv.cap + libcga::kTile - 1) / libcga::kTile);
    seg.out = p->lv;
    const uint32_t tiles = seg.num_tiles;
    const uint64_t keys = (uint64_t)tiles * libcga::kTile;
    void* scratch = dalloc(A, libcga::sort_scratch_bytes(keys, tiles, 1, false), s);
    if (scratch == nullptr) {
      rc = CGA_ERR_OOM;
    } else {
      const libcga::SortScratch sc = libcga::sort_scratch_carve(scratch, keys, tiles, 1, false);
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

int cga_nn_query(const cga_t* a, const float* d_q, uint64_t m, uint32_t* d_idx,
                 uint64_t* d_dist2, void* stream) {
  if (a == nullptr || (m > 0 && (d_q == nullptr || d_idx == nullptr || d_dist2 == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  if (m > libcga::kNnMaxQueries) return CGA_ERR_INVALID_ARG;
  if (m == 0) return CGA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
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
  if (p == nullptr) return;
  dfree(&p->alloc, p->has_alloc, p->mem, p->stream);
  delete p;
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
    default: return "unknown error";
  }
}

}  // extern "C"
