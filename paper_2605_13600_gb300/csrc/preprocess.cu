// preprocess.cu -- per-view projection of the Gaussians (paper Sec. 3).
//
// Standard 3DGS projection: camera-space mean, near-plane cull at z <= 0.2,
// Sigma3 = (R S)(R S)^T from the normalised quaternion and scales, EWA 2D
// covariance T Sigma3 T^T + 0.3 I with T = J Rv and the Jacobian J taken at
// the tangent clamped to 1.3x the half field of view, inverse covariance,
// radius ceil(3 sqrt(lambda_max)) with the 0.1 eigenvalue floor, and the
// 16x16 tile rectangle.
//
// This translation unit is compiled with --fmad=false: every expression is
// evaluated left to right in IEEE binary32 with each operation rounded, in the
// operation order written here, so the discrete outcomes (cull, radius,
// rectangle, depth) are reproducible on any IEEE binary32 machine.
//
// With depth slabs the kernel also resets the per-pixel slab state of the view
// and counts the listed Gaussians in a depth histogram (float bits >> 16: 128
// buckets per octave from 0.2 up); the last CTA to finish turns the histogram
// into the slab bounds (its quantiles) and clears it for the next view.
#include <math.h>

#include "scoup_internal.cuh"

namespace scoup {
namespace {

__device__ __forceinline__ int tile_clamp(float v, int g) {
  if (!(v > 0.0f)) return 0;
  if (v > (float)g) return g;
  return (int)v;
}

__device__ __forceinline__ int depth_bucket(uint32_t bits) {
  const uint32_t b = (bits >> 16) - kDepthBucketBase;  // bits >= those of 0.2f for every listed Gaussian
  return (int)min(b, (uint32_t)(kDepthBuckets - 1));
}

// Slab state of a view: the per-pixel transmittance records and the tile
// done flags start cleared (0 = untouched pixel, tile open).
struct SlabArgs {
  SlabPlan plan;
  uint32_t* dhist;
  float* pix_state;
  uint8_t* tile_done;
  int ntiles;
};

// Run by the last CTA of the projection: slab bounds at the plan's quantiles
// of the histogram; the histogram and the CTA counter are cleared.
__device__ void slab_bounds(const SlabArgs& sa, WsHeader* __restrict__ hdr, int slot) {
  constexpr int kPer = kDepthBuckets / 256;
  __shared__ uint32_t s_warp[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t c[kPer], sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) { c[q] = __ldcg(&sa.dhist[tid * kPer + q]); sum += c[q]; }
  uint32_t incl = sum;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0, total = 0;
  for (int w = 0; w < 8; ++w) { total += s_warp[w]; if (w < warp) wbase += s_warp[w]; }
  const uint32_t excl = wbase + incl - sum;
  if (tid == 0) hdr->slab_lo[slot][0] = 0u;
  for (int k = 0; k + 1 < sa.plan.nslabs; ++k) {
    // slab k + 1 starts after the bucket in which the running count reaches the target
    const uint32_t target = (uint32_t)ceilf(sa.plan.q[k] * (float)total);
    if (target == 0u) {
      if (tid == 0) hdr->slab_lo[slot][k + 1] = 0u;
    } else if (target > excl && target <= excl + sum) {
      uint32_t run = excl;
      int b = tid * kPer;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        run += c[q];
        if (run >= target) { b = tid * kPer + q; break; }
      }
      hdr->slab_lo[slot][k + 1] = (uint32_t)(b + 1 + kDepthBucketBase) << 16;
    }
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) sa.dhist[tid * kPer + q] = 0u;
  if (tid == 0) hdr->pp_blocks[slot] = 0u;
}

// Thread p projects Gaussian p of the spatially ordered copy; the record is
// stored at its original index, depth and rectangle in spatial order.
__global__ void __launch_bounds__(256) preprocess_kernel(
    const float* __restrict__ means, const float* __restrict__ scales,
    const float* __restrict__ quats, const float* __restrict__ opacity,
    const float* __restrict__ tau, const int32_t* __restrict__ orig, int64_t n, CamArgs cam,
    ProjRec* __restrict__ proj,
    uint32_t* __restrict__ depth_bits, ushort4* __restrict__ rects, WsHeader* __restrict__ hdr,
    int slot, SlabArgs sa) {
  __shared__ uint32_t s_hist[kDepthBuckets];
  const bool slabs = sa.plan.nslabs > 1;
  if (slabs) {
    for (int b = threadIdx.x; b < kDepthBuckets; b += blockDim.x) s_hist[b] = 0u;
    const int64_t nstate = (int64_t)sa.ntiles * (kTilePixels / 4);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nstate;
         i += (int64_t)gridDim.x * blockDim.x)
      reinterpret_cast<float4*>(sa.pix_state)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sa.ntiles;
         i += (int64_t)gridDim.x * blockDim.x)
      sa.tile_done[i] = 0;
    __syncthreads();
  }
  unsigned long long my_vis = 0, my_dups = 0;
  uint32_t my_dmin = 0xffffffffu, my_dmax = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    ushort4 rect = make_ushort4(0, 0, 0, 0);
    // every input of the Gaussian is loaded up front, so that all its loads
    // are in flight together (one memory round trip instead of two)
    const float m0 = means[3 * i], m1 = means[3 * i + 1], m2 = means[3 * i + 2];
    const float4 q = *reinterpret_cast<const float4*>(quats + 4 * i);
    const float s0 = scales[3 * i], s1 = scales[3 * i + 1], s2 = scales[3 * i + 2];
    const float op_i = opacity[i], tau_i = tau[i];
    const int32_t orig_i = orig[i];
    const float* W = cam.vm;
    float t0 = W[0] * m0 + W[1] * m1 + W[2] * m2 + W[3];
    float t1 = W[4] * m0 + W[5] * m1 + W[6] * m2 + W[7];
    float t2 = W[8] * m0 + W[9] * m1 + W[10] * m2 + W[11];
    depth_bits[i] = __float_as_uint(t2);
    if (t2 > 0.2f) {
      float qn = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
      float inv = 1.0f / sqrtf(qn);
      float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
      float R00 = 1.0f - 2.0f * (y * y + z * z);
      float R01 = 2.0f * (x * y - w * z);
      float R02 = 2.0f * (x * z + w * y);
      float R10 = 2.0f * (x * y + w * z);
      float R11 = 1.0f - 2.0f * (x * x + z * z);
      float R12 = 2.0f * (y * z - w * x);
      float R20 = 2.0f * (x * z - w * y);
      float R21 = 2.0f * (y * z + w * x);
      float R22 = 1.0f - 2.0f * (x * x + y * y);
      float M00 = R00 * s0, M01 = R01 * s1, M02 = R02 * s2;
      float M10 = R10 * s0, M11 = R11 * s1, M12 = R12 * s2;
      float M20 = R20 * s0, M21 = R21 * s1, M22 = R22 * s2;
      float S00 = M00 * M00 + M01 * M01 + M02 * M02;
      float S01 = M00 * M10 + M01 * M11 + M02 * M12;
      float S02 = M00 * M20 + M01 * M21 + M02 * M22;
      float S11 = M10 * M10 + M11 * M11 + M12 * M12;
      float S12 = M10 * M20 + M11 * M21 + M12 * M22;
      float S22 = M20 * M20 + M21 * M21 + M22 * M22;
      // S10 = S01, S20 = S02, S21 = S12 (each is the same rounded expression)

      float limx = 1.3f * (0.5f * (float)cam.width / cam.fx);
      float limy = 1.3f * (0.5f * (float)cam.height / cam.fy);
      float txz = t0 / t2, tyz = t1 / t2;
      float txc = fminf(limx, fmaxf(-limx, txz)) * t2;
      float tyc = fminf(limy, fmaxf(-limy, tyz)) * t2;
      float tz2 = t2 * t2;
      float j00 = cam.fx / t2;
      float j02 = -(cam.fx * txc) / tz2;
      float j11 = cam.fy / t2;
      float j12 = -(cam.fy * tyc) / tz2;
      float T00 = j00 * W[0] + j02 * W[8];
      float T01 = j00 * W[1] + j02 * W[9];
      float T02 = j00 * W[2] + j02 * W[10];
      float T10 = j11 * W[4] + j12 * W[8];
      float T11 = j11 * W[5] + j12 * W[9];
      float T12 = j11 * W[6] + j12 * W[10];
      float U00 = T00 * S00 + T01 * S01 + T02 * S02;
      float U01 = T00 * S01 + T01 * S11 + T02 * S12;
      float U02 = T00 * S02 + T01 * S12 + T02 * S22;
      float U10 = T10 * S00 + T11 * S01 + T12 * S02;
      float U11 = T10 * S01 + T11 * S11 + T12 * S12;
      float U12 = T10 * S02 + T11 * S12 + T12 * S22;
      float ca2 = U00 * T00 + U01 * T01 + U02 * T02 + 0.3f;
      float cb2 = U00 * T10 + U01 * T11 + U02 * T12;
      float cc2 = U10 * T10 + U11 * T11 + U12 * T12 + 0.3f;
      float det = ca2 * cc2 - cb2 * cb2;
      if (det > 0.0f) {
        float idet = 1.0f / det;
        float con_a = cc2 * idet, con_b = -cb2 * idet, con_c = ca2 * idet;
        float mid = 0.5f * (ca2 + cc2);
        float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
        float r = ceilf(3.0f * sqrtf(lam));
        float mx = cam.fx * txz + cam.cx - 0.5f;
        float my = cam.fy * tyz + cam.cy - 0.5f;
        int xlo = tile_clamp(floorf((mx - r) / 16.0f), cam.gx);
        int xhi = tile_clamp(floorf((mx + r + 15.0f) / 16.0f), cam.gx);
        int ylo = tile_clamp(floorf((my - r) / 16.0f), cam.gy);
        int yhi = tile_clamp(floorf((my + r + 15.0f) / 16.0f), cam.gy);
        if (xhi > xlo && yhi > ylo) {
          ProjRec pr;
          pr.a = make_float4(mx, my, -0.5f * con_a, -con_b);
          pr.b = make_float4(-0.5f * con_c, op_i, tau_i, log2f(op_i));
          proj[orig_i] = pr;
          // Binning lists only the tiles of the rectangle that also meet the
          // bounding box of the alpha >= 1/255 ellipse {d : power(d) >= tau}:
          // half-widths sqrt(-2 tau (A^-1)_xx), sqrt(-2 tau (A^-1)_yy) with
          // A = [[-2qa, -qb], [-qb, -2qc]], widened by 0.1% + 0.5 px so no
          // pixel centre that passes the alpha test is left out.
          int lx0 = xhi, lx1 = xlo, ly0 = yhi, ly1 = ylo;  // empty unless tau < 0
          if (tau_i < 0.0f) {
            const float A00 = con_a, A11 = con_c, A01 = con_b;  // = -2qa, -2qc, -qb
            const float detA = A00 * A11 - A01 * A01;
            const float ex = sqrtf(-2.0f * tau_i * A11 / detA) * 1.001f + 0.5f;
            const float ey = sqrtf(-2.0f * tau_i * A00 / detA) * 1.001f + 0.5f;
            lx0 = max(xlo, tile_clamp(floorf((mx - ex) / 16.0f), cam.gx));
            lx1 = min(xhi, tile_clamp(floorf((mx + ex) / 16.0f) + 1.0f, cam.gx));
            ly0 = max(ylo, tile_clamp(floorf((my - ey) / 16.0f), cam.gy));
            ly1 = min(yhi, tile_clamp(floorf((my + ey) / 16.0f) + 1.0f, cam.gy));
          }
          if (lx1 > lx0 && ly1 > ly0) {
            rect = make_ushort4((unsigned short)lx0, (unsigned short)ly0, (unsigned short)lx1,
                                (unsigned short)ly1);
            if (slabs) atomicAdd(&s_hist[depth_bucket(__float_as_uint(t2))], 1u);
          } else {
            rect = make_ushort4(0, 0, 0, 0);
          }
          my_vis += 1;
          my_dups += (unsigned long long)(xhi - xlo) * (unsigned long long)(yhi - ylo);
          my_dmin = min(my_dmin, __float_as_uint(t2));
          my_dmax = max(my_dmax, __float_as_uint(t2));
        }
      }
    }
    rects[i] = rect;
  }
  // block reduction of the counters
  for (int off = 16; off > 0; off >>= 1) {
    my_vis += __shfl_down_sync(0xffffffffu, my_vis, off);
    my_dups += __shfl_down_sync(0xffffffffu, my_dups, off);
    my_dmin = min(my_dmin, __shfl_down_sync(0xffffffffu, my_dmin, off));
    my_dmax = max(my_dmax, __shfl_down_sync(0xffffffffu, my_dmax, off));
  }
  __shared__ unsigned long long s_vis[8], s_dups[8];
  __shared__ uint32_t s_dmin[8], s_dmax[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { s_vis[warp] = my_vis; s_dups[warp] = my_dups; s_dmin[warp] = my_dmin; s_dmax[warp] = my_dmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += s_vis[k]; b += s_dups[k]; lo = min(lo, s_dmin[k]); hi = max(hi, s_dmax[k]);
    }
    if (a) {
      atomicAdd(&hdr->visible, a);
      atomicAdd(&hdr->duplicates, b);
      atomicMin(&hdr->drange[slot][0], lo);
      atomicMax(&hdr->drange[slot][1], hi);
    }
  }
  if (slabs) {
    __shared__ bool s_last;
    for (int b = threadIdx.x; b < kDepthBuckets; b += blockDim.x)
      if (s_hist[b]) atomicAdd(&sa.dhist[b], s_hist[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&hdr->pp_blocks[slot], 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      slab_bounds(sa, hdr, slot);
    }
  }
}

}  // namespace

cudaError_t launch_preprocess(const scoup_scene& sc, const CamArgs& cam, const UpliftWs& ws,
                              int slot, cudaStream_t st, const SlabPlan* plan) {
  if (sc.n <= 0) return cudaSuccess;
  int blocks = (int)((sc.n + 255) / 256);
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  SlabArgs sa;
  sa.plan.nslabs = 1;
  if (plan && plan->nslabs > 1) sa.plan = *plan;
  sa.dhist = ws.dhist;
  sa.pix_state = ws.pix_state;
  sa.tile_done = ws.tile_done;
  sa.ntiles = cam.gx * cam.gy;
  preprocess_kernel<<<blocks, 256, 0, st>>>(ws.sp.means, ws.sp.scales, ws.sp.quats, ws.sp.opacity,
                                            ws.sp.tau, ws.sp.orig, sc.n, cam, ws.proj, ws.depth, ws.rect,
                                            ws.hdr, slot, sa);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
