// The Value (attribute) array of a CGA (Sec. V): one row of uint8 channels
// per stored voxel, in CGA point order.
//   k_value_accumulate  each input point finds its voxel by the Sec. V-A
//                       lookup and adds its attributes (or offers its index)
//   k_value_finalize    per voxel: round-half-up mean (sum + k/2) / k of its
//                       k points (Sec. III-B: the colours of the points merged
//                       into one box are averaged), or the first point's row
//   k_merge_values      per voxel of a merge: the row of the input holding
//                       it; in both, the base's (a's) row or the average
//                       (a + b + 1) / 2 (Sec. II-A)
// Sums are integer atomics, 32-bit when no voxel can reach 2^32 (n * 255 <
// 2^32) and 64-bit otherwise, so every result is independent of the order in
// which points arrive.
#include <algorithm>

#include "k_common.cuh"

namespace libcga {

namespace {

template <typename S>
__global__ void k_value_accumulate(Levels a, ValueInput in, void* scratch) {
  const uint32_t h = (uint32_t)a.hdr->cnt[2];
  const uint32_t C = in.channels;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < in.n; i += stride) {
    const float* p = in.xyz + 3 * i;
    unsigned long long key;
    if (!point_key<unsigned long long>(__ldg(p), __ldg(p + 1), __ldg(p + 2), in.has_x != 0, in.X,
                                       in.scale, in.off, a.bits, key)) {
      continue;  // the build has recorded the non-finite point
    }
    bool found = false;
    const uint32_t v = rank_of_found(a, h, key, found);
    if (!found) {
      atomicOr(&a.hdr->err, kErrInternal);
      continue;
    }
    if (in.policy == kValueFirst) {
      atomicMin(static_cast<uint32_t*>(scratch) + v, (uint32_t)i);
    } else {
      S* s = static_cast<S*>(scratch) + (size_t)v * (C + 1);
      for (uint32_t c = 0; c < C; ++c) atomicAdd(s + c, (S)__ldg(in.attr + i * C + c));
      atomicAdd(s + C, (S)1);
    }
  }
}

template <typename S>
__global__ void k_value_finalize(Levels a, ValueInput in, const void* scratch, uint8_t* values) {
  const uint32_t u = (uint32_t)a.hdr->cnt[0];
  const uint32_t C = in.channels;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < u; v += stride) {
    if (in.policy == kValueFirst) {
      const uint32_t i = static_cast<const uint32_t*>(scratch)[v];
      for (uint32_t c = 0; c < C; ++c) {
        values[(size_t)v * C + c] = i < in.n ? __ldg(in.attr + (size_t)i * C + c) : (uint8_t)0;
      }
    } else {
      const S* s = static_cast<const S*>(scratch) + (size_t)v * (C + 1);
      const S k = s[C];
      for (uint32_t c = 0; c < C; ++c) {
        values[(size_t)v * C + c] = k > 0 ? (uint8_t)((s[c] + k / 2) / k) : (uint8_t)0;
      }
    }
  }
}

// One tile of the merged CGA's positions: the window is expanded into
// column and slab indices in shared memory, each voxel's key is looked up in
// both inputs (Sec. V-A) and its row follows the merge policy.
__global__ void __launch_bounds__(kThreads) k_merge_values(Levels m, Levels a, Levels b,
                                                           const uint8_t* __restrict__ va,
                                                           const uint8_t* __restrict__ vb,
                                                           uint32_t C, int policy,
                                                           uint8_t* __restrict__ vm) {
  __shared__ Window s_win;
  __shared__ uint16_t s_col[kTile], s_slab[kTile];
  __shared__ uint32_t s_warp[kWarps];
  const uint32_t u = (uint32_t)m.hdr->cnt[0];
  const uint32_t start = blockIdx.x * kTile;
  if (start >= u) return;
  const uint32_t cnt = min((uint32_t)kTile, u - start);
  if (threadIdx.x < 32) {
    const Window wv =
        warp_window_of(m, (uint32_t)m.hdr->cnt[1], (uint32_t)m.hdr->cnt[2], start, start + cnt - 1);
    if (threadIdx.x == 0) s_win = wv;
  }
  __syncthreads();
  const Window w = s_win;
  expand_window(m, w, start, cnt, s_col, s_slab, s_warp);
  const uint32_t bits = m.bits;
  const uint32_t ha = (uint32_t)a.hdr->cnt[2], hb = (uint32_t)b.hdr->cnt[2];
  for (uint32_t e = threadIdx.x; e < cnt; e += kThreads) {
    const uint32_t cr = s_col[e];
    const unsigned long long key =
        ((unsigned long long)__ldg(m.idx2 + w.x0 + s_slab[cr]) << (2 * bits)) |
        ((unsigned long long)__ldg(m.idx1 + w.c0 + cr) << bits) |
        (unsigned long long)__ldg(m.idx0 + start + e);
    bool fa = false, fb = false;
    const uint32_t ia = rank_of_found(a, ha, key, fa);
    const uint32_t ib = rank_of_found(b, hb, key, fb);
    uint8_t* out = vm + (size_t)(start + e) * C;
    for (uint32_t c = 0; c < C; ++c) {
      uint32_t v = 0;
      if (fa && fb) {
        const uint32_t x = __ldg(va + (size_t)ia * C + c), y = __ldg(vb + (size_t)ib * C + c);
        v = policy == kMergeBase ? x : (x + y + 1u) / 2u;
      } else if (fa) {
        v = __ldg(va + (size_t)ia * C + c);
      } else if (fb) {
        v = __ldg(vb + (size_t)ib * C + c);
      }
      out[c] = (uint8_t)v;
    }
  }
}

unsigned blocks_for(uint64_t work) {
  return (unsigned)std::min<uint64_t>((std::max<uint64_t>(work, 1) + 255) / 256,
                                      (uint64_t)device_sm_count() * 8);
}

}  // namespace

// 32-bit sums suffice while n points of at most 255 each cannot reach 2^32.
static bool narrow_sums(uint64_t n) { return n * 255ull < (1ull << 32); }

size_t value_scratch_bytes(uint64_t cap, uint32_t channels, int policy) {
  // sized for the wider sums: the count n is not known here
  return (size_t)std::max<uint64_t>(cap, 1) * (policy == kValueFirst ? 4 : 8 * (channels + 1));
}

cudaError_t run_build_values(const Levels& a, const ValueInput& in, void* scratch,
                             uint8_t* values, cudaStream_t stream) {
  const bool narrow = in.policy != kValueFirst && narrow_sums(in.n);
  const size_t bytes = narrow ? (size_t)std::max<uint64_t>(a.cap, 1) * 4 * (in.channels + 1)
                              : value_scratch_bytes(a.cap, in.channels, in.policy);
  cudaError_t e = cudaMemsetAsync(scratch, in.policy == kValueFirst ? 0xff : 0, bytes, stream);
  if (e != cudaSuccess) return e;
  if (narrow) {
    k_value_accumulate<uint32_t><<<blocks_for(in.n), 256, 0, stream>>>(a, in, scratch);
    k_value_finalize<uint32_t><<<blocks_for(a.cap), 256, 0, stream>>>(a, in, scratch, values);
  } else {
    k_value_accumulate<unsigned long long><<<blocks_for(in.n), 256, 0, stream>>>(a, in, scratch);
    k_value_finalize<unsigned long long><<<blocks_for(a.cap), 256, 0, stream>>>(a, in, scratch,
                                                                             values);
  }
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t run_merge_values(const Levels& m, const Levels& a, const Levels& b, const uint8_t* va,
                             const uint8_t* vb, uint32_t channels, int policy, uint8_t* vm,
                             cudaStream_t stream) {
  const uint64_t tiles = (m.cap + kTile - 1) / kTile;
  if (tiles == 0) return cudaSuccess;
  k_merge_values<<<(unsigned)tiles, kThreads, 0, stream>>>(m, a, b, va, vb, channels, policy, vm);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace libcga
