// CGA compaction of one tile of sorted keys (Sec. V arrays).
//
// Each key opens a new voxel when it differs from its predecessor, a new level-1
// group (an (x, y) column, or a U value of a projection) when key >> b differs,
// and a new level-2 group (an x slab) when key >> 2b differs.  The positions of
// the heads come from warp ballots, a block scan over the warps and a
// decoupled look-back over the tiles of the segment; each head then writes its
// coordinate and, for a group head, the pointer to its first child:
//   Y_pointer[column] = index of the column's first voxel,
//   X_pointer[slab]   = index of the slab's first column,
// which is the recurrence of Sec. V written as an exclusive prefix count.
// The last tile writes the sentinels Y_pointer[g] = u, X_pointer[h] = g and
// the level sizes.
#pragma once
#include "k_common.cuh"

namespace libcga {

struct CompactSmem {
  unsigned long long last[kWarps];
  uint32_t wcnt[kWarps][3];
  uint32_t tot[6];
};

// k: this thread's keys in warp-striped order (element e = w*32*kItems +
// i*32 + lane of the tile); elements e >= cnt are ignored.  prev/has_prev:
// the key just before the tile in the segment.
template <int LEVELS, typename K>
__device__ __forceinline__ void compact_tile(const K (&k)[kItems], uint32_t cnt, bool has_prev,
                                             K prev, uint32_t tile, uint32_t first_tile,
                                             bool last_tile, const Levels& out, uint32_t* clook,
                                             CompactSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t b = out.bits, sh1 = b, sh2 = 2 * b, m = (1u << b) - 1u;
  const uint32_t full = 0xffffffffu;
  if (lane == 31) sm.last[w] = (unsigned long long)k[kItems - 1];
  __syncthreads();
  const K rowprev = (w == 0) ? prev : (K)sm.last[w - 1];
  const bool hp0 = (w == 0) ? has_prev : true;
  uint32_t bU[kItems], bY[kItems], bX[kItems];
  uint32_t cU = 0, cY = 0, cX = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    K p = __shfl_up_sync(full, k[i], 1);
    K lastprev = rowprev;
    if (i > 0) lastprev = __shfl_sync(full, k[i > 0 ? i - 1 : 0], 31);
    if (lane == 0) p = lastprev;
    const bool hp = (lane == 0 && i == 0) ? hp0 : true;
    const uint32_t e = (uint32_t)(w * 32 * kItems + i * 32 + lane);
    const bool valid = e < cnt;
    const bool hu = valid && (!hp || k[i] != p);
    const bool hy = valid && (!hp || (k[i] >> sh1) != (p >> sh1));
    const bool hx = (LEVELS == 3) && valid && (!hp || (k[i] >> sh2) != (p >> sh2));
    bU[i] = __ballot_sync(full, hu);
    bY[i] = __ballot_sync(full, hy);
    bX[i] = (LEVELS == 3) ? __ballot_sync(full, hx) : 0u;
    cU += __popc(bU[i]);
    cY += __popc(bY[i]);
    cX += __popc(bX[i]);
  }
  if (lane == 0) {
    sm.wcnt[w][0] = cU;
    sm.wcnt[w][1] = cY;
    sm.wcnt[w][2] = cX;
  }
  __syncthreads();
  if (tid < LEVELS) {
    uint32_t run = 0;
    for (int x = 0; x < kWarps; ++x) {
      const uint32_t v = sm.wcnt[x][tid];
      sm.wcnt[x][tid] = run;
      run += v;
    }
    uint32_t* my = clook + (size_t)tile * 3 + tid;
    uint32_t excl = 0;
    if (tile == first_tile) {
      st_relaxed(my, kFlagInc | run);
    } else {
      st_relaxed(my, kFlagAgg | run);
      excl = lookback(clook + tid, 3, tile, first_tile, &out.hdr->err);
      st_relaxed(my, kFlagInc | ((excl + run) & kValMask));
    }
    sm.tot[tid] = excl;
    sm.tot[3 + tid] = excl + run;
  }
  __syncthreads();
  uint32_t rU = sm.tot[0] + sm.wcnt[w][0];
  uint32_t rY = sm.tot[1] + sm.wcnt[w][1];
  uint32_t rX = (LEVELS == 3) ? sm.tot[2] + sm.wcnt[w][2] : 0u;
  const uint32_t ltm = lanemask_lt();
  bool bad = false;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t pu = rU + __popc(bU[i] & ltm);
    const uint32_t py = rY + __popc(bY[i] & ltm);
    const uint32_t px = rX + __popc(bX[i] & ltm);
    if ((bU[i] >> lane) & 1u) {
      if (pu < out.cap) out.idx0[pu] = (uint16_t)((uint32_t)k[i] & m); else bad = true;
    }
    if ((bY[i] >> lane) & 1u) {
      if (py < out.cap1) {
        out.idx1[py] = (uint16_t)((uint32_t)(k[i] >> sh1) & m);
        out.ptr1[py] = pu;
      } else {
        bad = true;
      }
    }
    if (LEVELS == 3 && ((bX[i] >> lane) & 1u)) {
      if (px < out.cap2) {
        out.idx2[px] = (uint16_t)(uint32_t)(k[i] >> sh2);
        out.ptr2[px] = py;
      } else {
        bad = true;
      }
    }
    rU += __popc(bU[i]);
    rY += __popc(bY[i]);
    rX += __popc(bX[i]);
  }
  if (bad) atomicOr(&out.hdr->err, kErrInternal);
  if (last_tile && tid == 0) {
    const uint32_t U = sm.tot[3], G = sm.tot[4], H = sm.tot[5];
    if (G <= out.cap1) out.ptr1[G] = U;
    if (LEVELS == 3 && H <= out.cap2) out.ptr2[H] = G;
    out.hdr->cnt[0] = U;
    out.hdr->cnt[1] = G;
    out.hdr->cnt[2] = (LEVELS == 3) ? H : 0ull;
  }
}

}  // namespace libcga
