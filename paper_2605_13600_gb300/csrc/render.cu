// render.cu -- sparse coefficient rendering (paper Sec. 4.3, Eq. 7):
//   What(p) = sum_i e_i(p) w^_i,   e_i(p) = alpha_i(p) prod_{j<i} (1 - alpha_j(p)),
// with the K-sparse Top-K codes w^_i of the uplift, into a dense C-vector per
// pixel (unnormalised), plus the final transmittance and the list position of
// the last contributor (for the backward pass).
//
// This is the SIMT form, used for code rows wider than the tensor-core
// kernel takes (render_mma.cu).  One CTA per 16x16 tile.  The tile's key list is ordered window by window
// exactly as in the uplift (tile_order.cuh) and the window's records are
// staged in shared memory.  Each warp then takes pixels one at a time from a
// shared counter and walks the window 32 Gaussians per round: every lane
// evaluates one Gaussian (the same binary32 exponent and alpha test as the
// uplift), a warp product-scan of (1 - alpha) gives each lane its
// transmittance, the first lane that would bring T below 1e-4 ends the pixel,
// and the contributing lanes add e * val into the warp's dense C-vector in
// shared memory (K shared atomics each).  The window's Top-K codes are staged
// in shared memory with the records (atom ids as int16, entry-major so the
// lanes of a warp read consecutive words) whenever they fit, so the
// per-contribution reads never leave the SM.  A pixel's row is written once
// per window (coalesced); a pixel still open at the end of a window keeps its
// partial row in the output and resumes from it in the next window.  With
// bf16 output the row is rounded on every write, so a pixel spanning w
// windows carries at most w roundings (relative error <= w 2^-8).
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>

#include "tile_order.cuh"

namespace scoup {
namespace {

constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
using ROrder = OrderSmem<256, 10>;
constexpr size_t kStageMaxBytes = 48 * 1024;  // largest staged-code block

struct RenderSmem {
  ROrder ord;
  float4 rec_a[ROrder::kWin];
  float4 rec_b[ROrder::kWin];
  float T[kTilePixels];
  int last[kTilePixels];
  int done[kTilePixels];
  int next_pixel;
  unsigned long long cnt[2];
  // followed by kRWarps dense accumulators of C floats (dynamic)
};

// Each warp owns two copies of its dense row (one per half-warp), the second
// 16 words further so the halves' atomics fall on different banks (measured
// 5.5 -> 4.9 ms per 1920x1080 view; four copies cost a CTA per SM and lose).
__device__ __forceinline__ int row_stride(int C) { return 2 * C + 16; }
__device__ __forceinline__ float* warp_acc(RenderSmem& sm, int warp, int C) {
  return reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(&sm) + sizeof(RenderSmem)) + warp * row_stride(C);
}

// Staged codes of the window: values [K][kWin] then atom ids [K][kWin] (int16).
struct StagedCodes {
  float* val;
  short* idx;
};

__device__ __forceinline__ StagedCodes staged_codes(RenderSmem& sm, int C, int K) {
  float* v = warp_acc(sm, kRWarps, C);  // right after the warp rows
  StagedCodes sc;
  sc.val = v;
  sc.idx = reinterpret_cast<short*>(v + (size_t)K * ROrder::kWin);
  return sc;
}

// Walk the sorted window win[0..m) for pixel (px, py).  T, last and the
// accumulator carry the pixel's state; returns true once the pixel is done.
template <bool kStaged>
__device__ __forceinline__ bool walk_pixel(RenderSmem& sm, int m, int wbase, float fpx, float fpy,
                                           float& T, int& last, float* acc,
                                           const int32_t* __restrict__ topk_idx,
                                           const float* __restrict__ topk_val, const StagedCodes& sc,
                                           int K, int C, unsigned& n_eval, unsigned& n_contrib) {
  const int lane = threadIdx.x & 31;
  for (int w0 = 0; w0 < m; w0 += 32) {
    const int j = w0 + lane;
    const bool live = j < m;
    const int jj = live ? j : 0;
    const float4 a = sm.rec_a[jj];
    const float4 b = sm.rec_b[jj];
    const float dx = a.x - fpx, dy = a.y - fpy;
    const float power = fmaf(dx, fmaf(a.z, dx, __fmul_rn(a.w, dy)), __fmul_rn(__fmul_rn(b.x, dy), dy));
    const bool accept = live && power <= 0.0f && power >= b.z;
    const float alpha = accept ? fminf(0.99f, b.y * __expf(power)) : 0.0f;
    // inclusive product scan of (1 - alpha) over the lanes
    float P = 1.0f - alpha;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, P, off);
      if (lane >= off) P *= y;
    }
    float Pex = __shfl_up_sync(0xffffffffu, P, 1);
    if (lane == 0) Pex = 1.0f;
    const float Tl = T * Pex;        // transmittance in front of this Gaussian
    const float test = T * P;        // transmittance behind it
    const unsigned stopmask = __ballot_sync(0xffffffffu, accept && test < 1e-4f);
    const int first = stopmask ? __ffs(stopmask) - 1 : 32;
    const bool take = accept && lane < first;
    const unsigned livemask = __ballot_sync(0xffffffffu, live);
    const unsigned evalmask = first < 32 ? livemask & ((2u << first) - 1u) : livemask;
    n_eval += (lane == 0) ? __popc(evalmask) : 0u;
    const unsigned takemask = __ballot_sync(0xffffffffu, take);
    n_contrib += (lane == 0) ? __popc(takemask) : 0u;
    if (take) {
      const float e = alpha * Tl;
      if constexpr (kStaged) {
        for (int k = 0; k < K; ++k) {
          const int atom = sc.idx[k * ROrder::kWin + j];
          if (atom >= 0 && atom < C) atomicAdd(&acc[(lane >> 4) * (C + 16) + atom], e * sc.val[k * ROrder::kWin + j]);
        }
      } else {
        const int g = (int)(sm.ord.win[j] & 0xffffffffull);
        const int32_t* ci = topk_idx + (int64_t)g * K;
        const float* cv = topk_val + (int64_t)g * K;
        for (int k = 0; k < K; ++k) {
          const int atom = ci[k];
          if (atom >= 0 && atom < C) atomicAdd(&acc[(lane >> 4) * (C + 16) + atom], e * cv[k]);
        }
      }
    }
    if (takemask) last = wbase + w0 + (31 - __clz((int)takemask)) + 1;
    if (stopmask) {
      T = __shfl_sync(0xffffffffu, Tl, first);
      return true;
    }
    T = __shfl_sync(0xffffffffu, test, 31);
  }
  return false;
}

__device__ __forceinline__ void write_row(void* __restrict__ out, int64_t pix, bool bf16, const float* acc, int C) {
  const int lane = threadIdx.x & 31;
  if (bf16) {
    __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out) + pix * C;
    for (int c = lane; c < C; c += 32) o[c] = __float2bfloat16_rn(acc[c] + acc[C + 16 + c]);
  } else {
    float* o = reinterpret_cast<float*>(out) + pix * C;
    for (int c = lane; c < C; c += 32) o[c] = acc[c] + acc[C + 16 + c];
  }
}

// 4 CTAs per SM (64 registers): the walk is latency-bound and occupancy pays
// (measured 9.1 -> 5.5 ms per 1920x1080 view against 2 CTAs per SM; 5 spills more)
template <bool kStaged>
__global__ void __launch_bounds__(kRThreads, 4) render_tile_kernel(
    CamArgs cam, const ProjRec* __restrict__ proj, const unsigned long long* __restrict__ keys,
    const uint32_t* __restrict__ tile_start, int slot, const int32_t* __restrict__ topk_idx,
    const float* __restrict__ topk_val, int K, int C, void* __restrict__ out, int out_bf16, float* __restrict__ out_T,
    int32_t* __restrict__ out_last, WsHeader* __restrict__ hdr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RenderSmem& sm = *reinterpret_cast<RenderSmem*>(smem_raw);
  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tile % cam.gx, ty = tile / cam.gx;
  const uint32_t begin = tile_start[tile];
  const int n = (int)(tile_start[tile + 1] - begin);
  if (hdr->status & kStatCapacity) return;
  const unsigned long long* tkeys = keys + begin;
  float* acc = warp_acc(sm, warp, C);
  const StagedCodes sc = staged_codes(sm, C, K);

  for (int p = tid; p < kTilePixels; p += kRThreads) {
    const int px = tx * kTile + (p & (kTile - 1)), py = ty * kTile + (p >> 4);
    sm.T[p] = 1.0f;
    sm.last[p] = 0;
    sm.done[p] = !(px < cam.width && py < cam.height);
  }
  if (tid < 2) sm.cnt[tid] = 0ull;
  const OrderBuckets bk = order_buckets<ROrder>(hdr, slot);
  order_init(sm.ord, tkeys, n, bk);  // ends with a barrier
  unsigned n_eval = 0, n_contrib = 0;

  OrderState st;
  int wbase = 0;
  bool first_window = true;
  while (true) {
    const int m = n > 0 ? order_next_window(sm.ord, tkeys, n, bk, st, hdr) : 0;
    if (m < 0) break;
    if (m == 0 && !first_window) break;
    for (int j = tid; j < m; j += kRThreads) {
      const ProjRec pr = proj[(int)(sm.ord.win[j] & 0xffffffffull)];
      sm.rec_a[j] = pr.a;
      sm.rec_b[j] = pr.b;
    }
    if constexpr (kStaged) {
      // consecutive threads read consecutive entries of one Gaussian's code (coalesced)
      for (int t = tid; t < m * K; t += kRThreads) {
        const int j = t / K, k = t - j * K;
        const int64_t g = (int64_t)(sm.ord.win[j] & 0xffffffffull);
        const int atom = topk_idx[g * K + k];
        sc.idx[k * ROrder::kWin + j] = (short)(atom >= 0 && atom < C ? atom : -1);
        sc.val[k * ROrder::kWin + j] = topk_val[g * K + k];
      }
    }
    if (tid == 0) sm.next_pixel = 0;
    __syncthreads();
    while (true) {
      int p = 0;
      if (lane == 0) p = atomicAdd(&sm.next_pixel, 1);
      p = __shfl_sync(0xffffffffu, p, 0);
      if (p >= kTilePixels) break;
      if (sm.done[p]) continue;
      const int px = tx * kTile + (p & (kTile - 1)), py = ty * kTile + (p >> 4);
      const int64_t pix = (int64_t)py * cam.width + px;
      if (first_window) {
        for (int c = lane; c < C; c += 32) { acc[c] = 0.0f; acc[C + 16 + c] = 0.0f; }
      } else {
        // partial row of an earlier window
        for (int c = lane; c < C; c += 32) {
          acc[c] = out_bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(out)[pix * C + c])
                            : reinterpret_cast<const float*>(out)[pix * C + c];
          acc[C + 16 + c] = 0.0f;
        }
      }
      __syncwarp();
      float T = sm.T[p];
      int last = sm.last[p];
      const bool fin = m > 0 && walk_pixel<kStaged>(sm, m, wbase, (float)px, (float)py, T, last, acc, topk_idx,
                                                    topk_val, sc, K, C, n_eval, n_contrib);
      __syncwarp();
      write_row(out, pix, out_bf16 != 0, acc, C);
      if (lane == 0) {
        sm.T[p] = T;
        sm.last[p] = last;
        sm.done[p] = fin;
        if (out_T) out_T[(int64_t)py * cam.width + px] = T;
        if (out_last) out_last[(int64_t)py * cam.width + px] = last;
      }
      __syncwarp();
    }
    __syncthreads();
    first_window = false;
    wbase += m;
    if (m == 0) break;
    int open = 0;
    for (int p = tid; p < kTilePixels; p += kRThreads) open |= !sm.done[p];
    if (!__syncthreads_or(open)) break;
  }
  if (lane == 0) {
    atomicAdd(&sm.cnt[0], (unsigned long long)n_eval);
    atomicAdd(&sm.cnt[1], (unsigned long long)n_contrib);
  }
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&hdr->evaluated, sm.cnt[0]);
    atomicAdd(&hdr->contributions, sm.cnt[1]);
  }
}

}  // namespace

size_t staged_bytes(int K) { return (size_t)K * ROrder::kWin * (sizeof(float) + sizeof(short)); }

bool render_stages(int K) { return staged_bytes(K) <= kStageMaxBytes; }

// The tensor-core kernel (render_mma.cu) takes every shape it supports;
// SCOUP_RENDER_SIMT=1 in the environment selects this kernel instead.
bool render_uses_mma(int C, int K) {
  const char* f = getenv("SCOUP_RENDER_SIMT");
  return render_mma_supported(C, K) && !(f && f[0] == '1');
}

size_t render_smem_bytes(int C, int K) {
  if (render_uses_mma(C, K)) return render_mma_smem_bytes();
  return sizeof(RenderSmem) + sizeof(float) * (size_t)kRWarps * (size_t)(2 * C + 16) +
         (render_stages(K) ? staged_bytes(K) : 0);
}

cudaError_t launch_render_tiles(const CamArgs& cam, const UpliftWs& ws, int slot, const int32_t* topk_idx,
                                const float* topk_val, int K, int C, void* out, int out_bf16, float* out_T,
                                int32_t* out_last, cudaStream_t st) {
  if (render_uses_mma(C, K))
    return launch_render_mma(cam, ws, slot, topk_idx, topk_val, K, C, out, out_bf16, out_T, out_last, st);
  const int ntiles = cam.gx * cam.gy;
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = render_smem_bytes(C, K);
  const bool staged = render_stages(K);
  cudaError_t err = cudaFuncSetAttribute(staged ? render_tile_kernel<true> : render_tile_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (staged)
    render_tile_kernel<true><<<ntiles, kRThreads, smem, st>>>(cam, ws.proj, ws.keys, ws.tile_start, slot, topk_idx,
                                                              topk_val, K, C, out, out_bf16, out_T, out_last, ws.hdr);
  else
    render_tile_kernel<false><<<ntiles, kRThreads, smem, st>>>(cam, ws.proj, ws.keys, ws.tile_start, slot,
                                                               topk_idx, topk_val, K, C, out, out_bf16, out_T, out_last,
                                                               ws.hdr);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
