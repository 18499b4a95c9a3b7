// render_bwd.cu -- gradient of a loss through the sparse-code rendering
// (Eq. 7 with the compositing of Eq. 2) with respect to the Top-K values and
// the opacities.  For one pixel with contributions i = 1..m (front to back),
// g = dL/dWhat(p), gw_i = g . w^_i and S = sum_i e_i gw_i:
//   dL/dval_ik  += e_i g[idx_ik]
//   dL/dalpha_i  = T_i gw_i - (S - sum_{j<=i} e_j gw_j) / (1 - alpha_i)
//   dL/do_i     += dalpha_i/do_i dL/dalpha_i,   dalpha/do = G while o G < 0.99, else 0.
// Top-K indices, the alpha >= 1/255 test and the transmittance stop are held
// fixed (piecewise-constant decisions).
//
// Transmittance is recomputed, not stored: the tile's list is walked twice
// (window by window, same order as the forward), the first walk giving S per
// pixel, the second the gradients.  Per window, gradients of the window's
// Gaussians are summed over the tile's pixels in shared memory (entry-major,
// so a warp's lanes hit consecutive words) and flushed with one global atomic
// per (Gaussian, entry).  The window's Top-K codes are staged in shared
// memory with the records whenever they fit.
#include <math.h>

#include "tile_order.cuh"

namespace scoup {
namespace {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
using BOrder = OrderSmem<256, 10>;
constexpr size_t kBStageMaxBytes = 48 * 1024;

struct BwdSmem {
  BOrder ord;
  float4 rec_a[BOrder::kWin];
  float4 rec_b[BOrder::kWin];
  float T[kTilePixels];
  float S[kTilePixels];      // pass 1: running sum of e gw; pass 2: total
  float Sb[kTilePixels];     // pass 2: sum of e gw in front of the current position
  int done[kTilePixels];
  int next_pixel;
  // dynamic: g rows [kBWarps][C], dval [K][kWin], dop [kWin], staged codes
  // (values [K][kWin], atom ids [K][kWin] as int16)
};

struct BwdDyn {
  float* g;
  float* dval;
  float* dop;
  float* cval;
  short* cidx;
};

__device__ __forceinline__ BwdDyn bwd_dyn(BwdSmem& sm, int C, int K) {
  float* base = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(&sm) + sizeof(BwdSmem));
  BwdDyn d;
  d.g = base;
  d.dval = base + kBWarps * C;
  d.dop = d.dval + BOrder::kWin * K;
  d.cval = d.dop + BOrder::kWin;
  d.cidx = reinterpret_cast<short*>(d.cval + BOrder::kWin * K);
  return d;
}

// One pass of pixel (fpx, fpy) over window win[0..m).  pass 1 accumulates S;
// pass 2 accumulates the gradients of the window's Gaussians.
template <int kPass, bool kStaged>
__device__ __forceinline__ bool walk_bwd(BwdSmem& sm, const BwdDyn& dy, const float* gw_row, int m,
                                         float fpx, float fpy, float& T, float& S, float& Sb, float Stot,
                                         const int32_t* __restrict__ topk_idx, const float* __restrict__ topk_val,
                                         int K, int C) {
  const int lane = threadIdx.x & 31;
  for (int w0 = 0; w0 < m; w0 += 32) {
    const int j = w0 + lane;
    const bool live = j < m;
    const int jj = live ? j : 0;
    const float4 a = sm.rec_a[jj];
    const float4 b = sm.rec_b[jj];
    const float dx = a.x - fpx, dyy = a.y - fpy;
    const float power = fmaf(dx, fmaf(a.z, dx, __fmul_rn(a.w, dyy)), __fmul_rn(__fmul_rn(b.x, dyy), dyy));
    const bool accept = live && power <= 0.0f && power >= b.z;
    const float G = __expf(power);
    const float alpha = accept ? fminf(0.99f, b.y * G) : 0.0f;
    float P = 1.0f - alpha;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, P, off);
      if (lane >= off) P *= y;
    }
    float Pex = __shfl_up_sync(0xffffffffu, P, 1);
    if (lane == 0) Pex = 1.0f;
    const float Tl = T * Pex;
    const float test = T * P;
    const unsigned stopmask = __ballot_sync(0xffffffffu, accept && test < 1e-4f);
    const int first = stopmask ? __ffs(stopmask) - 1 : 32;
    const bool take = accept && lane < first;
    const float e = take ? alpha * Tl : 0.0f;
    const int gidx = (int)(sm.ord.win[jj] & 0xffffffffull);
    float gw = 0.0f;
    if (take) {
      if constexpr (kStaged) {
        for (int k = 0; k < K; ++k) {
          const int atom = dy.cidx[k * BOrder::kWin + j];
          if (atom >= 0) gw += dy.cval[k * BOrder::kWin + j] * gw_row[atom];
        }
      } else {
        const int32_t* ci = topk_idx + (int64_t)gidx * K;
        const float* cv = topk_val + (int64_t)gidx * K;
        for (int k = 0; k < K; ++k) {
          const int atom = ci[k];
          if (atom >= 0 && atom < C) gw += cv[k] * gw_row[atom];
        }
      }
    }
    const float eg = e * gw;
    // inclusive sum scan of e * gw over the lanes
    float incl = eg;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    if (kPass == 2 && take) {
      const float S_after = Stot - (Sb + incl);
      const float dLda = Tl * gw - S_after / (1.0f - alpha);
      const float dado = (b.y * G < 0.99f) ? G : 0.0f;
      atomicAdd(&dy.dop[j], dado * dLda);
      for (int k = 0; k < K; ++k) {
        int atom;
        if constexpr (kStaged) {
          atom = dy.cidx[k * BOrder::kWin + j];
        } else {
          atom = topk_idx[(int64_t)gidx * K + k];
          if (atom >= C) atom = -1;
        }
        if (atom >= 0) atomicAdd(&dy.dval[k * BOrder::kWin + j], e * gw_row[atom]);
      }
    }
    const float round_sum = __shfl_sync(0xffffffffu, incl, 31);
    if (kPass == 1) S += round_sum;
    else Sb += round_sum;
    if (stopmask) {
      T = __shfl_sync(0xffffffffu, Tl, first);
      return true;
    }
    T = __shfl_sync(0xffffffffu, test, 31);
  }
  return false;
}

// 4 CTAs per SM: with 256-key windows, staged codes and entry-major gradient
// sums, measured 4.9 -> 2.1 ms per 800x600 view (2 or 3 CTAs per SM: 2.4 ms)
template <bool kStaged>
__global__ void __launch_bounds__(kBThreads, 4) render_bwd_kernel(
    CamArgs cam, const ProjRec* __restrict__ proj, const unsigned long long* __restrict__ keys,
    const uint32_t* __restrict__ tile_start, int slot, const int32_t* __restrict__ topk_idx,
    const float* __restrict__ topk_val, int K, int C, const float* __restrict__ dL_dcodes,
    float* __restrict__ d_val, float* __restrict__ d_opacity, WsHeader* __restrict__ hdr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& sm = *reinterpret_cast<BwdSmem*>(smem_raw);
  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tile % cam.gx, ty = tile / cam.gx;
  const uint32_t begin = tile_start[tile];
  const int n = (int)(tile_start[tile + 1] - begin);
  if (n == 0) return;
  if (hdr->status & kStatCapacity) return;
  const unsigned long long* tkeys = keys + begin;
  const BwdDyn dy = bwd_dyn(sm, C, K);
  float* grow = dy.g + warp * C;
  const OrderBuckets bk = order_buckets<BOrder>(hdr, slot);
  order_init(sm.ord, tkeys, n, bk);

  for (int pass = 1; pass <= 2; ++pass) {
    for (int p = tid; p < kTilePixels; p += kBThreads) {
      const int px = tx * kTile + (p & (kTile - 1)), py = ty * kTile + (p >> 4);
      sm.T[p] = 1.0f;
      sm.Sb[p] = 0.0f;
      if (pass == 1) sm.S[p] = 0.0f;
      sm.done[p] = !(px < cam.width && py < cam.height);
    }
    __syncthreads();
    OrderState st;
    while (true) {
      const int m = order_next_window(sm.ord, tkeys, n, bk, st, hdr);
      if (m <= 0) break;
      for (int j = tid; j < m; j += kBThreads) {
        const ProjRec pr = proj[(int)(sm.ord.win[j] & 0xffffffffull)];
        sm.rec_a[j] = pr.a;
        sm.rec_b[j] = pr.b;
        if (pass == 2) {
          for (int k = 0; k < K; ++k) dy.dval[k * BOrder::kWin + j] = 0.0f;
          dy.dop[j] = 0.0f;
        }
      }
      if constexpr (kStaged) {
        for (int t = tid; t < m * K; t += kBThreads) {
          const int j = t / K, k = t - j * K;
          const int64_t g = (int64_t)(sm.ord.win[j] & 0xffffffffull);
          const int atom = topk_idx[g * K + k];
          dy.cidx[k * BOrder::kWin + j] = (short)(atom >= 0 && atom < C ? atom : -1);
          dy.cval[k * BOrder::kWin + j] = topk_val[g * K + k];
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
        const float* g = dL_dcodes + ((int64_t)py * cam.width + px) * C;
        for (int c = lane; c < C; c += 32) grow[c] = g[c];
        __syncwarp();
        float T = sm.T[p], S = sm.S[p], Sb = sm.Sb[p];
        const bool fin = pass == 1
            ? walk_bwd<1, kStaged>(sm, dy, grow, m, (float)px, (float)py, T, S, Sb, 0.0f, topk_idx, topk_val, K, C)
            : walk_bwd<2, kStaged>(sm, dy, grow, m, (float)px, (float)py, T, S, Sb, sm.S[p], topk_idx, topk_val,
                                   K, C);
        if (lane == 0) {
          sm.T[p] = T;
          if (pass == 1) sm.S[p] = S;
          sm.Sb[p] = Sb;
          sm.done[p] = fin;
        }
        __syncwarp();
      }
      __syncthreads();
      if (pass == 2) {
        // flush the window's per-Gaussian gradient sums
        for (int j = tid; j < m; j += kBThreads) {
          const int64_t gi = (int64_t)(sm.ord.win[j] & 0xffffffffull);
          const float dop = dy.dop[j];
          if (dop != 0.0f) atomicAdd(&d_opacity[gi], dop);
          for (int k = 0; k < K; ++k) {
            const float v = dy.dval[k * BOrder::kWin + j];
            if (v != 0.0f) atomicAdd(&d_val[gi * K + k], v);
          }
        }
        __syncthreads();
      }
      int open = 0;
      for (int p = tid; p < kTilePixels; p += kBThreads) open |= !sm.done[p];
      if (!__syncthreads_or(open)) break;
    }
    __syncthreads();
  }
}

}  // namespace

bool bwd_stages(int K) { return (size_t)K * BOrder::kWin * (sizeof(float) + sizeof(short)) <= kBStageMaxBytes; }

size_t render_bwd_smem_bytes(int C, int K) {
  return sizeof(BwdSmem) + sizeof(float) * ((size_t)kBWarps * C + (size_t)BOrder::kWin * (K + 1)) +
         (bwd_stages(K) ? (size_t)K * BOrder::kWin * (sizeof(float) + sizeof(short)) : 0);
}

cudaError_t launch_render_bwd(const CamArgs& cam, const UpliftWs& ws, int slot, const int32_t* topk_idx,
                              const float* topk_val, int K, int C, const float* dL_dcodes, float* d_val,
                              float* d_opacity, cudaStream_t st) {
  const int ntiles = cam.gx * cam.gy;
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = render_bwd_smem_bytes(C, K);
  const bool staged = bwd_stages(K);
  cudaError_t err = cudaFuncSetAttribute(staged ? render_bwd_kernel<true> : render_bwd_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (staged)
    render_bwd_kernel<true><<<ntiles, kBThreads, smem, st>>>(cam, ws.proj, ws.keys, ws.tile_start, slot, topk_idx,
                                                             topk_val, K, C, dL_dcodes, d_val, d_opacity, ws.hdr);
  else
    render_bwd_kernel<false><<<ntiles, kBThreads, smem, st>>>(cam, ws.proj, ws.keys, ws.tile_start, slot,
                                                              topk_idx, topk_val, K, C, dL_dcodes, d_val,
                                                              d_opacity, ws.hdr);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
