// Served loop over device-resident CGAs: continuous batching with admission by
// device-memory footprint.
//
// A host scheduler thread owns `slots` CUDA streams.  Whenever a slot is idle
// and requests are pending, it forms one batch from the head of the queue.
// Requests join in arrival order while their estimated footprint fits the
// memory budget still free, up to `max_batch` requests.  All NN requests of the
// batch go into one segmented NN launch set; all merge+project requests into
// one batched merge and one batched projection.  The batch is queued on the
// slot's stream and an event is recorded behind it.  While it runs, requests
// that arrive meanwhile are batched onto the other slots, so their work overlaps
// on the GPU.  When a batch's event completes, its footprint is released and
// its requests are reported done with host timestamps (arrival, start, done).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/cga.h"
#include "cga_impl.h"

namespace libcga {
void handle_parts(const cga_t* a, Levels* lv, cga_grid* g);
void rebind_stream(cga_t* a, cga2d_t* p, cudaStream_t s);
}

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Pending {
  uint64_t ticket;
  cga_request req;
  uint64_t t_submit;
  uint64_t footprint;
};

struct InFlight {
  cudaEvent_t done = nullptr;
  std::vector<Pending> reqs;
  std::vector<cga_t*> merged;
  std::vector<cga2d_t*> projected;
  std::vector<int> status;
  uint64_t footprint = 0;
  uint64_t t_start = 0;
  bool busy = false;
};

uint64_t align256(uint64_t v) { return (v + 255) & ~(uint64_t)255; }

}  // namespace

struct cga_server {
  std::vector<const cga_t*> pool;
  std::vector<uint64_t> pool_cap;
  std::vector<uint32_t> pool_bits;
  cga_server_config cfg{};
  cga_allocator alloc{};
  bool has_alloc = false;
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<InFlight> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> pending;
  std::vector<cga_completion> done;
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, completed = 0;
  uint64_t reserved = 0;  // footprint of in-flight batches
  bool stop = false;
  std::thread worker;
  std::condition_variable done_cv;
};

namespace {

// Device bytes a request needs while it runs (scratch and outputs).
uint64_t footprint_of(const cga_server* s, const cga_request& r) {
  if (r.kind == CGA_REQ_NN) {
    const uint64_t tiles = (r.m + libcga::kTile - 1) / libcga::kTile;
    return libcga::nn_scratch_bytes((uint32_t)tiles, 1);
  }
  const uint64_t cap = s->pool_cap[r.a] + s->pool_cap[r.b];
  // merged CGA (<= 14 B per point) + merge scratch + projection output and its
  // re-key sort scratch (two 4-byte key buffers + look-back words)
  return align256(14 * cap + 4096) + align256(cap / 256 + 4096) + align256(6 * cap + 4096) +
         align256(8 * cap + (cap / libcga::kTile + 1) * 6 * 1024 + 65536);
}

void launch_batch(cga_server* s, InFlight& slot, cudaStream_t st) {
  const cga_allocator* A = s->has_alloc ? &s->alloc : nullptr;
  std::vector<const cga_t*> nn_a;
  std::vector<cga_queries> nn_q;
  std::vector<const cga_t*> ma, mb;
  std::vector<int> planes;
  std::vector<size_t> nn_ix, mp_ix;
  slot.status.assign(slot.reqs.size(), CGA_OK);
  slot.merged.assign(slot.reqs.size(), nullptr);
  slot.projected.assign(slot.reqs.size(), nullptr);
  for (size_t i = 0; i < slot.reqs.size(); ++i) {
    const cga_request& r = slot.reqs[i].req;
    if (r.kind == CGA_REQ_NN) {
      nn_a.push_back(s->pool[r.a]);
      nn_q.push_back(cga_queries{r.d_q, r.m, r.d_idx, r.d_dist2});
      nn_ix.push_back(i);
    } else {
      ma.push_back(s->pool[r.a]);
      mb.push_back(s->pool[r.b]);
      planes.push_back(r.plane);
      mp_ix.push_back(i);
    }
  }
  if (!nn_a.empty()) {
    const int rc = cga_nn_query_batch(nn_a.data(), nn_q.data(), (uint32_t)nn_a.size(), A, st);
    if (rc != CGA_OK) {
      for (size_t k : nn_ix) slot.status[k] = rc;
    }
  }
  if (!ma.empty()) {
    std::vector<cga_t*> m(ma.size(), nullptr);
    int rc = cga_merge_batch(ma.data(), mb.data(), (uint32_t)ma.size(), A, st, m.data());
    std::vector<cga2d_t*> p(ma.size(), nullptr);
    if (rc == CGA_OK) {
      std::vector<const cga_t*> mc(m.begin(), m.end());
      rc = cga_project_batch(mc.data(), planes.data(), (uint32_t)ma.size(), A, st, p.data());
      if (rc != CGA_OK) {
        for (cga_t* h : m) cga_free(h);
        std::fill(m.begin(), m.end(), nullptr);
      }
    }
    for (size_t k = 0; k < mp_ix.size(); ++k) {
      slot.status[mp_ix[k]] = rc;
      slot.merged[mp_ix[k]] = m[k];
      slot.projected[mp_ix[k]] = p[k];
    }
  }
  cudaEventRecord(slot.done, st);
}

void worker_main(cga_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (true) {
    bool progress = false;
    // completions
    for (size_t k = 0; k < s->slots.size(); ++k) {
      InFlight& sl = s->slots[k];
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      const uint64_t t = now_ns();
      for (size_t i = 0; i < sl.reqs.size(); ++i) {
        cga_completion c{};
        c.ticket = sl.reqs[i].ticket;
        c.status = q == cudaSuccess ? sl.status[i] : CGA_ERR_CUDA;
        c.t_submit_ns = sl.reqs[i].t_submit;
        c.t_start_ns = sl.t_start;
        c.t_done_ns = t;
        c.merged = sl.merged[i];
        c.projected = sl.projected[i];
        // the batch is complete: later waits and frees of the results go to
        // the default stream, which outlives the server's streams
        libcga::rebind_stream(c.merged, c.projected, nullptr);
        s->done.push_back(c);
      }
      if (q != cudaSuccess) cudaGetLastError();
      s->completed += sl.reqs.size();
      s->reserved -= sl.footprint;
      sl.reqs.clear();
      sl.busy = false;
      progress = true;
    }
    if (progress) s->done_cv.notify_all();
    // admission: one batch per idle slot
    for (size_t k = 0; k < s->slots.size() && !s->pending.empty(); ++k) {
      InFlight& sl = s->slots[k];
      if (sl.busy) continue;
      uint64_t fp = 0;
      while (!s->pending.empty() && sl.reqs.size() < s->cfg.max_batch) {
        const Pending& p = s->pending.front();
        if (s->reserved + fp + p.footprint > s->cfg.memory_budget && !sl.reqs.empty()) break;
        if (s->reserved + fp + p.footprint > s->cfg.memory_budget && s->reserved > 0) break;
        fp += p.footprint;
        sl.reqs.push_back(p);
        s->pending.pop_front();
      }
      if (sl.reqs.empty()) break;
      sl.footprint = fp;
      s->reserved += fp;
      sl.busy = true;
      sl.t_start = now_ns();
      InFlight* slp = &sl;
      cudaStream_t st = s->streams[k];
      lock.unlock();
      launch_batch(s, *slp, st);
      lock.lock();
      progress = true;
    }
    if (s->stop && s->pending.empty()) {
      bool idle = true;
      for (const InFlight& sl : s->slots) idle = idle && !sl.busy;
      if (idle) break;
    }
    if (!progress) {
      s->cv.wait_for(lock, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

extern "C" {

uint64_t cga_now_ns(void) { return now_ns(); }

int cga_server_create(const cga_t* const* pool, uint32_t count, const cga_server_config* cfg,
                      const cga_allocator* A, cga_server_t** out) {
  if (pool == nullptr || count == 0 || cfg == nullptr || out == nullptr || cfg->slots == 0 ||
      cfg->slots > 64 || cfg->max_batch == 0 || cfg->memory_budget == 0) {
    return CGA_ERR_INVALID_ARG;
  }
  if (A != nullptr && (A->alloc == nullptr || A->free == nullptr)) return CGA_ERR_INVALID_ARG;
  cga_server* s = new (std::nothrow) cga_server();
  if (s == nullptr) return CGA_ERR_OOM;
  s->cfg = *cfg;
  if (A != nullptr) {
    s->alloc = *A;
    s->has_alloc = true;
  }
  cudaGetDevice(&s->device);
  for (uint32_t i = 0; i < count; ++i) {
    if (pool[i] == nullptr) {
      delete s;
      return CGA_ERR_INVALID_ARG;
    }
    cga_sizes sz{};
    const int rc = cga_info(pool[i], &sz);  // waits for the pool's builds
    if (rc != CGA_OK) {
      delete s;
      return rc;
    }
    libcga::Levels lv{};
    cga_grid g{};
    libcga::handle_parts(pool[i], &lv, &g);
    s->pool.push_back(pool[i]);
    s->pool_cap.push_back(lv.cap);
    s->pool_bits.push_back(g.bits);
  }
  s->streams.resize(cfg->slots, nullptr);
  s->slots.resize(cfg->slots);
  for (uint32_t k = 0; k < cfg->slots; ++k) {
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->slots[k].done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (auto st : s->streams) if (st) cudaStreamDestroy(st);
      for (auto& sl : s->slots) if (sl.done) cudaEventDestroy(sl.done);
      delete s;
      return CGA_ERR_CUDA;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return CGA_OK;
}

int cga_server_submit(cga_server_t* s, const cga_request* r, uint64_t* ticket) {
  if (s == nullptr || r == nullptr) return CGA_ERR_INVALID_ARG;
  const uint32_t n = (uint32_t)s->pool.size();
  if (r->kind == CGA_REQ_NN) {
    if (r->a >= n || r->m > libcga::kNnMaxQueries ||
        (r->m > 0 && (r->d_q == nullptr || r->d_idx == nullptr || r->d_dist2 == nullptr))) {
      return CGA_ERR_INVALID_ARG;
    }
  } else if (r->kind == CGA_REQ_MERGE_PROJECT) {
    if (r->a >= n || r->b >= n || r->plane < CGA_PLANE_XY || r->plane > CGA_PLANE_YZ) {
      return CGA_ERR_INVALID_ARG;
    }
    cga_grid ga{}, gb{};
    libcga::Levels la{}, lb{};
    libcga::handle_parts(s->pool[r->a], &la, &ga);
    libcga::handle_parts(s->pool[r->b], &lb, &gb);
    if (ga.bits != gb.bits || std::memcmp(&ga.scale, &gb.scale, sizeof(float)) != 0 ||
        std::memcmp(ga.offset, gb.offset, sizeof(ga.offset)) != 0) {
      return CGA_ERR_GRID_MISMATCH;
    }
  } else {
    return CGA_ERR_INVALID_ARG;
  }
  const uint64_t fp = footprint_of(s, *r);
  if (fp > s->cfg.memory_budget) return CGA_ERR_OOM;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return CGA_ERR_INVALID_ARG;
    Pending p{s->next_ticket++, *r, now_ns(), fp};
    if (ticket != nullptr) *ticket = p.ticket;
    s->pending.push_back(p);
    ++s->submitted;
  }
  s->cv.notify_one();
  return CGA_OK;
}

int cga_server_poll(cga_server_t* s, cga_completion* out, uint32_t max, uint32_t* n) {
  if (s == nullptr || n == nullptr || (max > 0 && out == nullptr)) return CGA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  const uint32_t k = (uint32_t)std::min<size_t>(max, s->done.size());
  for (uint32_t i = 0; i < k; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *n = k;
  return CGA_OK;
}

int cga_server_drain(cga_server_t* s) {
  if (s == nullptr) return CGA_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  s->done_cv.wait(lock, [s] { return s->completed == s->submitted; });
  return CGA_OK;
}

void cga_server_free(cga_server_t* s) {
  if (s == nullptr) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& c : s->done) {
    cga_free(c.merged);
    cga2d_free(c.projected);
  }
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto& sl : s->slots) cudaEventDestroy(sl.done);
  delete s;
}

}  // extern "C"
