// Launch-shape tuning of the sort and merge kernels: a process-wide table
// keyed by (grid bits, power-of-two bucket of the element count), and the
// autotuner that fills an entry by timing the candidates on the caller's own
// cloud.  The kernels compute the same result under every shape; only their
// speed differs.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "cga.h"
#include "cga_impl.h"

namespace libcga {

namespace {

constexpr int kBuckets = 65;  // bit length of n: 0..64
constexpr uint32_t kSet = 1u << 31;

// Packed entry: radix bits | (sort_threads / 256) << 4 | log2(merge_half) << 8.
std::atomic<uint32_t> g_table[17][kBuckets];

int bucket_of(uint64_t n) { return n == 0 ? 0 : 64 - __builtin_clzll(n); }

uint32_t pack(const Tuning& t) {
  uint32_t lg = 0;
  while ((1u << lg) < t.merge_half) ++lg;
  return kSet | t.radix_bits | ((t.sort_threads / 256u) << 4) | (lg << 8);
}

Tuning unpack(uint32_t v) {
  return Tuning{v & 15u, ((v >> 4) & 15u) * 256u, 1u << ((v >> 8) & 31u)};
}

}  // namespace

bool tuning_valid(const Tuning& t) {
  const bool sort_ok = (t.radix_bits == 8 && (t.sort_threads == 256 || t.sort_threads == 512)) ||
                       (t.radix_bits == 9 && t.sort_threads == 512);
  const bool merge_ok = t.merge_half == 512 || t.merge_half == 1024 || t.merge_half == 2048;
  return sort_ok && merge_ok;
}

Tuning tuning_for(uint32_t bits, uint64_t n) {
  if (bits < 1 || bits > 16) return kDefaultTuning;
  const uint32_t v = g_table[bits][bucket_of(n)].load(std::memory_order_relaxed);
  return (v & kSet) ? unpack(v) : kDefaultTuning;
}

void tuning_store(uint32_t bits, uint64_t n, const Tuning* t) {
  if (bits < 1 || bits > 16) return;
  g_table[bits][bucket_of(n)].store(t != nullptr ? pack(*t) : 0u, std::memory_order_relaxed);
}

}  // namespace libcga

namespace {

libcga::Tuning from_abi(const cga_tuning& t) {
  return libcga::Tuning{t.radix_bits, t.sort_threads, t.merge_half};
}

cga_tuning to_abi(const libcga::Tuning& t) {
  cga_tuning o{};
  o.radix_bits = t.radix_bits;
  o.sort_threads = t.sort_threads;
  o.merge_half = t.merge_half;
  return o;
}

// Least time of `reps` runs of fn (each bracketed by events on s), after one
// untimed warm-up run.
template <typename F>
int time_min(F fn, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* best) {
  int rc = fn();
  if (rc != CGA_OK) return rc;
  float b = -1.0f;
  for (int r = 0; r < reps; ++r) {
    if (cudaEventRecord(e0, s) != cudaSuccess) return CGA_ERR_CUDA;
    rc = fn();
    if (rc != CGA_OK) return rc;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      return CGA_ERR_CUDA;
    }
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return CGA_ERR_CUDA;
    if (b < 0.0f || ms < b) b = ms;
  }
  *best = b;
  return CGA_OK;
}

}  // namespace

extern "C" {

int cga_tuning_set(uint32_t bits, uint64_t n, const cga_tuning* t) {
  if (bits < 1 || bits > 16) return CGA_ERR_INVALID_ARG;
  if (t != nullptr && !libcga::tuning_valid(from_abi(*t))) return CGA_ERR_INVALID_ARG;
  if (t == nullptr) {
    libcga::tuning_store(bits, n, nullptr);
  } else {
    const libcga::Tuning v = from_abi(*t);
    libcga::tuning_store(bits, n, &v);
  }
  return CGA_OK;
}

int cga_tuning_get(uint32_t bits, uint64_t n, cga_tuning* out) {
  if (out == nullptr || bits < 1 || bits > 16) return CGA_ERR_INVALID_ARG;
  *out = to_abi(libcga::tuning_for(bits, n));
  return CGA_OK;
}

int cga_autotune(const float* d_xyz, uint64_t n, const cga_grid* g, cga_tuning* chosen,
                 float* times_ms, void* stream) {
  if (d_xyz == nullptr || g == nullptr || chosen == nullptr || n < 2 || n > CGA_MAX_POINTS ||
      g->bits < 1 || g->bits > 16) {
    return CGA_ERR_INVALID_ARG;
  }
  static const libcga::Tuning sort_cand[CGA_TUNE_SORT_CANDIDATES] = {
      {8u, 256u, 0u}, {8u, 512u, 0u}, {9u, 512u, 0u}};
  static const uint32_t merge_cand[CGA_TUNE_MERGE_CANDIDATES] = {512u, 1024u, 2048u};
  const uint32_t bits = g->bits;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const libcga::Tuning before = libcga::tuning_for(bits, n);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess
               ? CGA_OK
               : CGA_ERR_CUDA;
  libcga::Tuning best = before;
  float best_ms = -1.0f;
  // the sort shape, on a build of the whole cloud
  for (int k = 0; k < CGA_TUNE_SORT_CANDIDATES && rc == CGA_OK; ++k) {
    libcga::Tuning t = sort_cand[k];
    t.merge_half = before.merge_half;
    libcga::tuning_store(bits, n, &t);
    float ms = 0.0f;
    rc = time_min(
        [&]() {
          cga_t* a = nullptr;
          const int r = cga_build(d_xyz, n, g, nullptr, nullptr, stream, &a);
          if (a != nullptr) cga_free(a);
          return r;
        },
        2, s, e0, e1, &ms);
    if (rc != CGA_OK) break;
    if (times_ms) times_ms[k] = ms;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best.radix_bits = t.radix_bits;
      best.sort_threads = t.sort_threads;
    }
  }
  // the merge-path partition, on the merge of the cloud's two halves
  cga_t* A = nullptr;
  cga_t* B = nullptr;
  if (rc == CGA_OK) {
    libcga::tuning_store(bits, n, &best);
    const uint64_t h = n / 2;
    rc = cga_build(d_xyz, h, g, nullptr, nullptr, stream, &A);
    if (rc == CGA_OK) rc = cga_build(d_xyz + 3 * h, n - h, g, nullptr, nullptr, stream, &B);
  }
  best_ms = -1.0f;
  uint32_t best_half = best.merge_half;
  for (int k = 0; k < CGA_TUNE_MERGE_CANDIDATES && rc == CGA_OK; ++k) {
    libcga::Tuning t = best;
    t.merge_half = merge_cand[k];
    libcga::tuning_store(bits, n, &t);
    float ms = 0.0f;
    rc = time_min(
        [&]() {
          cga_t* m = nullptr;
          const int r = cga_merge(A, B, nullptr, stream, &m);
          if (m != nullptr) cga_free(m);
          return r;
        },
        2, s, e0, e1, &ms);
    if (rc != CGA_OK) break;
    if (times_ms) times_ms[CGA_TUNE_SORT_CANDIDATES + k] = ms;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best_half = t.merge_half;
    }
  }
  best.merge_half = best_half;
  if (A != nullptr) cga_free(A);
  if (B != nullptr) cga_free(B);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != CGA_OK) {
    libcga::tuning_store(bits, n, &before);
    return rc;
  }
  libcga::tuning_store(bits, n, &best);
  *chosen = to_abi(best);
  return CGA_OK;
}

int cga_pipeline_autotune(const cga_pipeline_item* items, uint32_t count, cga_tuning* chosen,
                          float* times_ms, void* stream) {
  if (items == nullptr || count == 0 || chosen == nullptr) return CGA_ERR_INVALID_ARG;
  uint32_t bits = 1;
  uint64_t n = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (items[i].grid.bits < 1 || items[i].grid.bits > 16) return CGA_ERR_INVALID_ARG;
    bits = std::max(bits, items[i].grid.bits);
    n = std::max<uint64_t>(n, items[i].n);
  }
  static const libcga::Tuning sort_cand[CGA_TUNE_SORT_CANDIDATES] = {
      {8u, 256u, 0u}, {8u, 512u, 0u}, {9u, 512u, 0u}};
  static const uint32_t merge_cand[CGA_TUNE_MERGE_CANDIDATES] = {512u, 1024u, 2048u};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const libcga::Tuning before = libcga::tuning_for(bits, n);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess
               ? CGA_OK
               : CGA_ERR_CUDA;
  // one pipeline per candidate: its first graph launch captures, the timed
  // ones replay
  auto time_shape = [&](const libcga::Tuning& t, float* ms) {
    libcga::tuning_store(bits, n, &t);
    cga_pipeline_t* p = nullptr;
    int r = cga_pipeline_create(items, count, nullptr, stream, &p);
    if (r == CGA_OK) r = time_min([&]() { return cga_pipeline_run_graph(p, stream); }, 2, s, e0, e1, ms);
    if (p != nullptr) {
      if (cudaStreamSynchronize(s) != cudaSuccess && r == CGA_OK) r = CGA_ERR_CUDA;
      cga_pipeline_free(p);
    }
    return r;
  };
  libcga::Tuning best = before;
  float best_ms = -1.0f;
  for (int k = 0; k < CGA_TUNE_SORT_CANDIDATES && rc == CGA_OK; ++k) {
    libcga::Tuning t = sort_cand[k];
    t.merge_half = before.merge_half;
    float ms = 0.0f;
    rc = time_shape(t, &ms);
    if (rc != CGA_OK) break;
    if (times_ms) times_ms[k] = ms;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  best_ms = -1.0f;
  uint32_t best_half = best.merge_half;
  for (int k = 0; k < CGA_TUNE_MERGE_CANDIDATES && rc == CGA_OK; ++k) {
    libcga::Tuning t = best;
    t.merge_half = merge_cand[k];
    float ms = 0.0f;
    rc = time_shape(t, &ms);
    if (rc != CGA_OK) break;
    if (times_ms) times_ms[CGA_TUNE_SORT_CANDIDATES + k] = ms;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best_half = t.merge_half;
    }
  }
  best.merge_half = best_half;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != CGA_OK) {
    libcga::tuning_store(bits, n, &before);
    return rc;
  }
  libcga::tuning_store(bits, n, &best);
  *chosen = to_abi(best);
  return CGA_OK;
}

}  // extern "C"
