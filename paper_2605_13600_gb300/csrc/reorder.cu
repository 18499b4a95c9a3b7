// reorder.cu -- one-time spatial reordering of the scene for binning locality.
//
// Gaussians are grouped by the 3D Morton code of a 32^3 grid over the
// bounding box of their means (a counting sort), and the scene arrays are
// gathered into that order in the workspace.  Gaussians that are close in 3D
// project close together in every view, so a binning CTA's chunk of
// consecutive Gaussians covers a compact set of tiles and writes long
// contiguous runs of keys.  The original index travels with every Gaussian:
// keys, records and accumulator rows stay addressed by it, so no result
// depends on this order.  The per-Gaussian alpha-threshold exponent tau is
// computed here as well.
#include <math.h>

#include "scoup_internal.cuh"

namespace scoup {
namespace {

constexpr int kCells = 1 << 15;  // 32^3 Morton cells

__device__ __forceinline__ uint32_t ordered_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_ordered(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 5 bits -> every third bit
  v &= 0x1fu;
  v = (v | (v << 8)) & 0x0100f00fu;
  v = (v | (v << 4)) & 0x010c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void bbox_kernel(const float* __restrict__ means, int64_t n, WsHeader* __restrict__ hdr) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const uint32_t u = ordered_bits(means[3 * i + a]);
      lo[a] = min(lo[a], u);
      hi[a] = max(hi[a], u);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int off = 16; off > 0; off >>= 1) {
      lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
      hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&hdr->bbox[a][0], lo[a]);
      atomicMax(&hdr->bbox[a][1], hi[a]);
    }
  }
}

__global__ void cell_kernel(const float* __restrict__ means, int64_t n, const WsHeader* __restrict__ hdr,
                            uint32_t* __restrict__ cell, uint32_t* __restrict__ cnt) {
  float lo[3], scale[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = from_ordered(hdr->bbox[a][0]);
    const float ext = from_ordered(hdr->bbox[a][1]) - lo[a];
    scale[a] = ext > 0.0f ? 32.0f / ext : 0.0f;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float f = (means[3 * i + a] - lo[a]) * scale[a];
      q[a] = f > 0.0f ? (uint32_t)min(f, 31.0f) : 0u;
    }
    const uint32_t c = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    cell[i] = c;
    atomicAdd(&cnt[c], 1u);
  }
}

// Exclusive scan of the cell counts into start[], cursors zeroed (one CTA).
__global__ void __launch_bounds__(1024) cell_scan_kernel(const uint32_t* __restrict__ cnt,
                                                         uint32_t* __restrict__ start,
                                                         uint32_t* __restrict__ cur) {
  constexpr int kPer = kCells / 1024;
  __shared__ uint32_t s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t c[kPer], sum = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) { c[k] = cnt[tid * kPer + k]; sum += c[k]; }
  uint32_t incl = sum;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = s_warp[lane];
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t run = (warp ? s_warp[warp - 1] : 0u) + incl - sum;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    start[tid * kPer + k] = run;
    cur[tid * kPer + k] = 0u;
    run += c[k];
  }
}

__global__ void gather_kernel(const float* __restrict__ means, const float* __restrict__ scales,
                              const float* __restrict__ quats, const float* __restrict__ opacity,
                              int64_t n, const uint32_t* __restrict__ cell,
                              const uint32_t* __restrict__ start, uint32_t* __restrict__ cur,
                              SceneP sp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = cell[i];
    const int64_t p = (int64_t)start[c] + atomicAdd(&cur[c], 1u);
    sp.means[3 * p] = means[3 * i];
    sp.means[3 * p + 1] = means[3 * i + 1];
    sp.means[3 * p + 2] = means[3 * i + 2];
    sp.scales[3 * p] = scales[3 * i];
    sp.scales[3 * p + 1] = scales[3 * i + 1];
    sp.scales[3 * p + 2] = scales[3 * i + 2];
    *reinterpret_cast<float4*>(sp.quats + 4 * p) = *reinterpret_cast<const float4*>(quats + 4 * i);
    const float o = opacity[i];
    sp.opacity[p] = o;
    sp.orig[p] = (int32_t)i;
    // smallest binary32 tau with o * exp(tau) >= 1/255, i.e. ceil_f(-log(255 o))
    const double t = o > 0.0f ? -log(255.0 * (double)o) : INFINITY;
    float th = (float)t;
    if ((double)th < t) th = nextafterf(th, INFINITY);
    sp.tau[p] = th;
  }
}

__global__ void init_header_kernel(WsHeader* __restrict__ hdr) {
  const int t = threadIdx.x;
  if (t < 3) { hdr->bbox[t][0] = 0xffffffffu; hdr->bbox[t][1] = 0u; }
  if (t < 4) { hdr->drange[t][0] = 0xffffffffu; hdr->drange[t][1] = 0u; }
}

int grid_for(int64_t n, int per_sm) {
  int64_t b = (n + 255) / 256;
  if (b > num_sms() * per_sm) b = num_sms() * per_sm;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

size_t reorder_scratch_bytes() { return sizeof(uint32_t) * (size_t)(3 * kCells); }

cudaError_t launch_reorder(const scoup_scene& sc, const UpliftWs& ws, cudaStream_t st) {
  init_header_kernel<<<1, 32, 0, st>>>(ws.hdr);
  g_launches += 1;
  if (sc.n <= 0) return cudaGetLastError();
  uint32_t* cnt = ws.cells_scratch;
  uint32_t* start = cnt + kCells;
  uint32_t* cur = start + kCells;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kCells, st);
  if (e != cudaSuccess) return e;
  bbox_kernel<<<grid_for(sc.n, 4), 256, 0, st>>>(sc.means, sc.n, ws.hdr);
  cell_kernel<<<grid_for(sc.n, 8), 256, 0, st>>>(sc.means, sc.n, ws.hdr, ws.cell, cnt);
  cell_scan_kernel<<<1, 1024, 0, st>>>(cnt, start, cur);
  gather_kernel<<<grid_for(sc.n, 8), 256, 0, st>>>(sc.means, sc.scales, sc.quats, sc.opacity, sc.n,
                                                   ws.cell, start, cur, ws.sp);
  g_launches += 4;
  return cudaGetLastError();
}

}  // namespace scoup
