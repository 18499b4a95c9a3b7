// loss.cu -- the L2 loss between decoded features and per-pixel region
// targets, and its gradient (the loss of the differentiable sparse render).
//
// The target of pixel p is the decoded code of its region,
// F*(p) = sum_j v_j C[j] over the s entries (j, v_j) of code_{r(p)} (the
// region codes of Eq. 5, decoded with the codebook C of Eq. 8).  The loss is
// L = sum_p |F(p) - F*(p)|^2 over labelled pixels, and dL/dF(p) = 2 (F - F*).
// A first kernel decodes every region's target once (R x D floats, resident
// in L2), a second one streams the pixels: one warp per pixel row of D
// features, lanes over the features.
#include <cuda_bf16.h>

#include "scoup_internal.cuh"

namespace scoup {
namespace {

// F*_r[d] = sum_j v_j C[j][d] for every region r (one warp per region).
__global__ void __launch_bounds__(256) region_target_kernel(const int32_t* __restrict__ ci,
                                                            const float* __restrict__ cv, int R, int s,
                                                            const float* __restrict__ codebook, int C, int D,
                                                            float* __restrict__ target, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += warps) {
    for (int d = lane; d < D; d += 32) {
      float acc = 0.0f;
      for (int e = 0; e < s; ++e) {
        const int j = ci[r * s + e];
        if (j >= C) { atomicOr(status, kStatDeviceCheck); continue; }
        if (j >= 0) acc = fmaf(cv[r * s + e], codebook[(int64_t)j * D + d], acc);
      }
      target[r * D + d] = acc;
    }
  }
}

template <bool kInBF16, bool kOutBF16>
__global__ void __launch_bounds__(256) l2_grad_kernel(const void* __restrict__ F, int64_t P, int D,
                                                      const int32_t* __restrict__ rmap, int R,
                                                      const float* __restrict__ target, void* __restrict__ dF,
                                                      double* __restrict__ loss, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  double part = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
    int r = rmap[p];
    if (r >= R) {
      if (lane == 0) atomicOr(status, kStatDeviceCheck);
      r = -1;
    }
    float sq = 0.0f;
    for (int d = lane; d < D; d += 32) {
      float f;
      if constexpr (kInBF16) f = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(F)[p * D + d]);
      else f = reinterpret_cast<const float*>(F)[p * D + d];
      // unlabelled pixels (region -1) have no target: no loss, no gradient
      const float diff = r >= 0 ? f - target[(int64_t)r * D + d] : 0.0f;
      sq = fmaf(diff, diff, sq);
      if constexpr (kOutBF16) reinterpret_cast<__nv_bfloat16*>(dF)[p * D + d] = __float2bfloat16_rn(2.0f * diff);
      else reinterpret_cast<float*>(dF)[p * D + d] = 2.0f * diff;
    }
    part += (double)sq;
  }
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if (lane == 0 && loss && part != 0.0) atomicAdd(loss, part);
}

int blocks_for_warps(int64_t rows) {
  int64_t b = (rows + 7) / 8;
  if (b > num_sms() * 16) b = num_sms() * 16;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_region_targets(const int32_t* ci, const float* cv, int R, int s, const float* codebook, int C,
                                  int D, float* target, int* status, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  region_target_kernel<<<blocks_for_warps(R), 256, 0, st>>>(ci, cv, R, s, codebook, C, D, target, status);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_l2_grad(const void* F, int F_bf16, int64_t P, int D, const int32_t* rmap, int R,
                           const float* target, void* dF, int dF_bf16, double* loss, int* status, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  const int b = blocks_for_warps(P);
  if (F_bf16 && dF_bf16) l2_grad_kernel<true, true><<<b, 256, 0, st>>>(F, P, D, rmap, R, target, dF, loss, status);
  else if (F_bf16) l2_grad_kernel<true, false><<<b, 256, 0, st>>>(F, P, D, rmap, R, target, dF, loss, status);
  else if (dF_bf16) l2_grad_kernel<false, true><<<b, 256, 0, st>>>(F, P, D, rmap, R, target, dF, loss, status);
  else l2_grad_kernel<false, false><<<b, 256, 0, st>>>(F, P, D, rmap, R, target, dF, loss, status);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
