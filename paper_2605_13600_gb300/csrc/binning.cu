// binning.cu -- tile binning of one view's projected Gaussians.
//
// Every visible Gaussian is listed in each 16x16 tile of its rectangle (the
// 3DGS rule: membership is tile-granular).  The per-tile lists hold 64-bit
// keys (depth bits << 32 | Gaussian id); they are left unordered here and
// ordered front to back (depth, then id) inside the tile kernel.
//
// Counting and filling are privatised per CTA in shared memory (one counter
// per tile of the view) so that global atomics are one per (CTA, tile) rather
// than one per (Gaussian, tile); views with more tiles than fit fall back to
// global atomics.
#include "scoup_internal.cuh"

namespace scoup {
namespace {

constexpr int kBinThreads = 512;
constexpr int kSmemTilesMax = 24 * 1024;  // 2 x 96 KB of counters at most

template <bool kSmem>
__global__ void __launch_bounds__(kBinThreads) count_kernel(const ushort4* __restrict__ rects,
                                                            int64_t n, int64_t chunk, int ntiles,
                                                            int gx, uint32_t* __restrict__ tile_count) {
  extern __shared__ uint32_t s_cnt[];
  if (kSmem) {
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s_cnt[t] = 0;
    __syncthreads();
  }
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const ushort4 r = rects[i];
    for (int ty = r.y; ty < r.w; ++ty)
      for (int tx = r.x; tx < r.z; ++tx) {
        const int t = ty * gx + tx;
        if (kSmem) atomicAdd(&s_cnt[t], 1u);
        else atomicAdd(&tile_count[t], 1u);
      }
  }
  if (kSmem) {
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
      if (s_cnt[t]) atomicAdd(&tile_count[t], s_cnt[t]);
  }
}

// Exclusive scan of the tile counts (one CTA), capacity check, and reset of
// the counters and fill cursors for the next view.
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* __restrict__ tile_count,
                                                    uint32_t* __restrict__ tile_start,
                                                    uint32_t* __restrict__ tile_fill, int ntiles,
                                                    int64_t capacity, WsHeader* __restrict__ hdr) {
  __shared__ uint32_t s_warp[32];
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    const int t = base + threadIdx.x;
    uint32_t v = t < ntiles ? tile_count[t] : 0u;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const unsigned long long carry = s_carry;
    const uint32_t excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0u);
    if (t < ntiles) {
      tile_start[t] = (uint32_t)(carry + excl);
      tile_count[t] = 0u;
      tile_fill[t] = 0u;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = carry + excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long total = s_carry;
    tile_start[ntiles] = (uint32_t)total;
    if ((long long)total > capacity || total > 0xffffffffull) atomicOr(&hdr->status, kStatCapacity);
    atomicMax(&hdr->max_dups_view, (int)min(total, 0x7fffffffull));
  }
}

template <bool kSmem>
__global__ void __launch_bounds__(kBinThreads) fill_kernel(
    const ushort4* __restrict__ rects, const uint32_t* __restrict__ depth, int64_t n, int64_t chunk,
    int ntiles, int gx, const uint32_t* __restrict__ tile_start, uint32_t* __restrict__ tile_fill,
    unsigned long long* __restrict__ keys, const WsHeader* __restrict__ hdr) {
  extern __shared__ uint32_t s_mem[];
  uint32_t* s_cnt = s_mem;
  uint32_t* s_base = s_mem + ntiles;
  if (hdr->status & kStatCapacity) return;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  if (kSmem) {
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s_cnt[t] = 0;
    __syncthreads();
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const ushort4 r = rects[i];
      for (int ty = r.y; ty < r.w; ++ty)
        for (int tx = r.x; tx < r.z; ++tx) atomicAdd(&s_cnt[ty * gx + tx], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
      const uint32_t c = s_cnt[t];
      if (c) s_base[t] = tile_start[t] + atomicAdd(&tile_fill[t], c);
      s_cnt[t] = 0;
    }
    __syncthreads();
  }
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const ushort4 r = rects[i];
    if (r.z <= r.x) continue;
    const unsigned long long key = ((unsigned long long)depth[i] << 32) | (unsigned long long)i;
    for (int ty = r.y; ty < r.w; ++ty)
      for (int tx = r.x; tx < r.z; ++tx) {
        const int t = ty * gx + tx;
        uint32_t pos;
        if (kSmem) pos = s_base[t] + atomicAdd(&s_cnt[t], 1u);
        else pos = tile_start[t] + atomicAdd(&tile_fill[t], 1u);
        keys[pos] = key;
      }
  }
}

}  // namespace

cudaError_t launch_binning(const CamArgs& cam, int64_t n, const UpliftWs& ws, cudaStream_t st) {
  const int ntiles = cam.gx * cam.gy;
  if (n > 0) {
    const int64_t chunk = 4096;
    const int blocks = (int)((n + chunk - 1) / chunk);
    if (ntiles <= kSmemTilesMax) {
      const size_t smem = sizeof(uint32_t) * (size_t)ntiles;
      cudaFuncSetAttribute(count_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      count_kernel<true><<<blocks, kBinThreads, smem, st>>>(ws.rect, n, chunk, ntiles, cam.gx,
                                                           ws.tile_count);
    } else {
      count_kernel<false><<<blocks, kBinThreads, 0, st>>>(ws.rect, n, chunk, ntiles, cam.gx,
                                                         ws.tile_count);
    }
  }
  scan_kernel<<<1, 1024, 0, st>>>(ws.tile_count, ws.tile_start, ws.tile_fill, ntiles,
                                  ws.dup_capacity, ws.hdr);
  if (n > 0) {
    const int64_t chunk = 4096;
    const int blocks = (int)((n + chunk - 1) / chunk);
    if (ntiles <= kSmemTilesMax) {
      const size_t smem = 2 * sizeof(uint32_t) * (size_t)ntiles;
      cudaFuncSetAttribute(fill_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      fill_kernel<true><<<blocks, kBinThreads, smem, st>>>(ws.rect, ws.depth, n, chunk, ntiles,
                                                          cam.gx, ws.tile_start, ws.tile_fill,
                                                          ws.keys, ws.hdr);
    } else {
      fill_kernel<false><<<blocks, kBinThreads, 0, st>>>(ws.rect, ws.depth, n, chunk, ntiles,
                                                        cam.gx, ws.tile_start, ws.tile_fill,
                                                        ws.keys, ws.hdr);
    }
  }
  g_launches += n > 0 ? 3 : 1;
  return cudaGetLastError();
}

}  // namespace scoup
