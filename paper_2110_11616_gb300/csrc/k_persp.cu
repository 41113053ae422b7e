// Perspective projection of a CGA onto an image (Eq. 5-6): every stored voxel
// is moved to the eye's frame, rotated about the y axis (Eq. 6) and divided by
// its depth onto the plane at distance D (Eq. 5); each pixel keeps the voxel
// of least depth, ties to the smaller CGA index.
//   k_perspective         one tile of voxels per block (window expanded in
//                         shared memory), one 64-bit atomic minimum per voxel
//                         on (depth bits << 32 | index): a positive float's
//                         bits order like the float, so the minimum is the
//                         nearest voxel and then the smallest index
//   k_perspective_finish  the packed z-buffer to index and depth images
// The arithmetic is one IEEE operation per step in a fixed order (no
// contraction), so the image is the same on every run and device.
#include <algorithm>

#include "k_common.cuh"

namespace libcga {

namespace {

__global__ void __launch_bounds__(kThreads) k_perspective(Levels a, Camera cam,
                                                          unsigned long long* zbuf) {
  __shared__ Window s_win;
  __shared__ uint16_t s_col[kTile], s_slab[kTile];
  __shared__ uint32_t s_warp[kWarps];
  const uint32_t u = (uint32_t)a.hdr->cnt[0];
  const uint32_t start = blockIdx.x * kTile;
  if (start >= u) return;
  const uint32_t cnt = min((uint32_t)kTile, u - start);
  if (threadIdx.x < 32) {
    const Window wv =
        warp_window_of(a, (uint32_t)a.hdr->cnt[1], (uint32_t)a.hdr->cnt[2], start, start + cnt - 1);
    if (threadIdx.x == 0) s_win = wv;
  }
  __syncthreads();
  const Window w = s_win;
  expand_window(a, w, start, cnt, s_col, s_slab, s_warp);
  const float half_w = (float)cam.W * 0.5f, half_h = (float)cam.H * 0.5f;
  const float neg_sin = -cam.sin_t;
  for (uint32_t e = threadIdx.x; e < cnt; e += kThreads) {
    const uint32_t cr = s_col[e];
    const float sx = __fsub_rn((float)__ldg(a.idx2 + w.x0 + s_slab[cr]), cam.eye[0]);
    const float sy = __fsub_rn((float)__ldg(a.idx1 + w.c0 + cr), cam.eye[1]);
    const float sz = __fsub_rn((float)__ldg(a.idx0 + start + e), cam.eye[2]);
    const float xr = __fmaf_rn(cam.cos_t, sx, __fmul_rn(neg_sin, sz));
    const float zr = __fmaf_rn(cam.sin_t, sx, __fmul_rn(cam.cos_t, sz));
    if (!(zr > 0.0f)) continue;  // at or behind the eye
    const float px = __fdiv_rn(__fmul_rn(cam.D, xr), zr);
    const float py = __fdiv_rn(__fmul_rn(cam.D, sy), zr);
    const float fu = floorf(__fadd_rn(px, half_w)), fv = floorf(__fadd_rn(py, half_h));
    if (!(fu >= 0.0f && fu < (float)cam.W && fv >= 0.0f && fv < (float)cam.H)) continue;
    const size_t pix = (size_t)fv * cam.W + (size_t)fu;
    atomicMin(zbuf + pix,
              ((unsigned long long)__float_as_uint(zr) << 32) | (unsigned long long)(start + e));
  }
}

__global__ void k_perspective_finish(const unsigned long long* __restrict__ zbuf, uint64_t npix,
                                     uint32_t* __restrict__ index, float* __restrict__ depth) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < npix; i += stride) {
    const unsigned long long v = zbuf[i];
    index[i] = (uint32_t)v;
    depth[i] = v == ~0ull ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(v >> 32));
  }
}

}  // namespace

cudaError_t run_perspective(const Levels& a, const Camera& cam, unsigned long long* zbuf,
                            uint32_t* index, float* depth, cudaStream_t stream) {
  const uint64_t npix = (uint64_t)cam.W * cam.H;
  cudaError_t e = cudaMemsetAsync(zbuf, 0xff, npix * sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = (a.cap + kTile - 1) / kTile;
  if (tiles > 0) k_perspective<<<(unsigned)tiles, kThreads, 0, stream>>>(a, cam, zbuf);
  const unsigned blocks = (unsigned)std::min<uint64_t>((npix + 255) / 256,
                                                       (uint64_t)device_sm_count() * 8);
  k_perspective_finish<<<blocks, 256, 0, stream>>>(zbuf, npix, index, depth);
  count_launch(tiles > 0 ? 2 : 1);
  return cudaGetLastError();
}

}  // namespace libcga
