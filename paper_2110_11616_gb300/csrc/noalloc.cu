// cga_nn_query_noalloc: exact NN queries that allocate no memory.
//
// Some callers cannot allocate device memory at the moment they query: code
// running under a fixed memory budget that was reserved up front, real-time
// loops that must not call cudaMalloc (it can synchronize the device and its
// latency is unbounded), and hosts whose allocator is owned by another
// framework.  This entry point takes the scratch of the query sort (keys,
// digit histograms, look-back words, descriptor tables) from one file-scope
// __device__ array of fixed size instead of allocating it.  The caller still
// provides the CGA, the queries and the outputs.
#include <mutex>

#include "../../include/cga.h"
#include "cga_impl.h"

namespace libcga {
void handle_parts(const cga_t* a, Levels* lv, cga_grid* g);
void nn_attach(const cga_t* a, NnSeg& seg);
}

namespace {

// Scratch for CGA_NOALLOC_MAX_QUERIES queries: two key buffers of 8 MiB, the
// look-back words of four passes over 256 tiles, histograms and tables.
constexpr size_t kStaticScratchBytes = (size_t)18 << 20;
static __device__ __align__(256) unsigned char g_nn_scratch[kStaticScratchBytes];

// Device address of g_nn_scratch on the current device, looked up once per
// device (host code only holds a stand-in for the symbol; the kernels need the
// address).  nullptr when the lookup fails.
void* scratch_address() {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_nn_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace

extern "C" int cga_nn_query_noalloc(const cga_t* a, const float* d_q, uint64_t m, uint32_t* d_idx,
                                    uint64_t* d_dist2, void* stream) {
  if (a == nullptr || (m > 0 && (d_q == nullptr || d_idx == nullptr || d_dist2 == nullptr))) {
    return CGA_ERR_INVALID_ARG;
  }
  if (m > CGA_NOALLOC_MAX_QUERIES) return CGA_ERR_CAPACITY;
  if (m == 0) return CGA_OK;
  const uint32_t tiles = (uint32_t)((m + libcga::kTile - 1) / libcga::kTile);
  if (libcga::nn_scratch_bytes(tiles, 1) > kStaticScratchBytes) return CGA_ERR_INTERNAL;
  void* scratch = scratch_address();
  if (scratch == nullptr) return CGA_ERR_CUDA;
  libcga::Levels lv{};
  cga_grid g{};
  libcga::handle_parts(a, &lv, &g);
  libcga::NnSeg seg{};
  seg.a = lv;
  seg.scale = g.scale;
  for (int k = 0; k < 3; ++k) seg.off[k] = g.offset[k];
  seg.q = d_q;
  seg.m = (uint32_t)m;
  seg.idx = d_idx;
  seg.d2 = reinterpret_cast<unsigned long long*>(d_dist2);
  seg.tile_base = 0;
  seg.num_tiles = tiles;
  // the search structures cga_nn_prepare_levels built on `a`, as cga_nn_query uses them
  libcga::nn_attach(a, seg);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const libcga::NnTables t = libcga::nn_tables(scratch, tiles, 1);
  cudaError_t e = libcga::nn_upload_one(seg, t, s);
  if (e == cudaSuccess) e = libcga::run_nn_device(1, tiles, t, s, 1u << libcga::nn_kind(seg));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CGA_ERR_CUDA;
  }
  return CGA_OK;
}
