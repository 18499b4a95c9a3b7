// topk.cu -- Top-K consensus filter + L1 normalisation (paper Eq. 6, Alg. 1)
// and the per-code Top-K of Algorithm 1 for codes with more than K entries.
//
// One warp per accumulator row.  Lane l holds entries l, l+32, l+64, ... in
// registers; each of the K rounds picks the largest remaining positive entry
// (ties to the lower atom index): every lane offers its best remaining entry,
// one warp reduction takes the maximum of the offered values' bit patterns
// (positive floats order as their bits) and a second the lowest atom index
// among the lanes that offer that maximum.  The row is read once from HBM
// (coalesced).
// With a compensation array (the compensated uplift) each entry is the FP32
// sum of the running sum and its compensation.  Optionally the same pass
// writes the entropy of the row's coefficient distribution,
// H = -sum p log p with p = w / sum w over the positive entries (0 for an
// empty row), computed as log S - (sum w log w) / S; the per-entry logarithms
// use the fast intrinsic (absolute error about 1e-6, so H is off by at most
// that much: far inside the FP32 tolerance of the entropy).
#include "scoup_internal.cuh"

namespace scoup {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int VPL>
__global__ void __launch_bounds__(256) topk_kernel(const float* __restrict__ acc, const float* __restrict__ comp,
                                                   int64_t n, int C, int64_t ld, int K,
                                                   int32_t* __restrict__ idx, float* __restrict__ val,
                                                   float* __restrict__ entropy) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
    const float* a = acc + row * ld;
    float v[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
      const int j = lane + 32 * k;
      v[k] = j < C ? (comp ? __fadd_rn(a[j], comp[row * ld + j]) : a[j]) : 0.0f;
    }
    if (entropy) {
      float S = 0.0f, WL = 0.0f;
#pragma unroll
      for (int k = 0; k < VPL; ++k)
        if (v[k] > 0.0f) {
          S += v[k];
          WL = fmaf(v[k], __logf(v[k]), WL);
        }
      for (int off = 16; off > 0; off >>= 1) {
        S += __shfl_xor_sync(kFull, S, off);
        WL += __shfl_xor_sync(kFull, WL, off);
      }
      if (lane == 0) entropy[row] = S > 0.0f ? fmaxf(0.0f, logf(S) - WL / S) : 0.0f;
    }
    unsigned taken = 0u;
    float sum = 0.0f;
    int32_t* orow_i = idx + row * K;
    float* orow_v = val + row * K;
    int r = 0;
    for (; r < K; ++r) {
      float bv = 0.0f;
      int bj = 0x7fffffff;
#pragma unroll
      for (int k = 0; k < VPL; ++k) {
        if (!((taken >> k) & 1u) && v[k] > bv) { bv = v[k]; bj = lane + 32 * k; }
      }
      const unsigned mb = __reduce_max_sync(kFull, __float_as_uint(bv));
      if (mb == 0u) break;  // no positive entry left
      bj = __reduce_min_sync(kFull, __float_as_uint(bv) == mb ? bj : 0x7fffffff);
      bv = __uint_as_float(mb);
      if ((bj & 31) == lane) taken |= 1u << (bj >> 5);
      if (lane == 0) { orow_i[r] = bj; orow_v[r] = bv; }
      sum += bv;
    }
    __syncwarp();
    for (int k = lane; k < K; k += 32) {
      if (k < r) {
        orow_v[k] = orow_v[k] / sum;
      } else {
        orow_i[k] = -1;
        orow_v[k] = 0.0f;
      }
    }
    __syncwarp();
  }
}

// Per code row: keep the K largest entries (ties to the lower atom id), pad -1.
__global__ void code_topk_kernel(const int32_t* __restrict__ ci, const float* __restrict__ cv,
                                 int64_t R, int s, int K, int32_t* __restrict__ co,
                                 float* __restrict__ cvo) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* a = ci + r * s;
    const float* b = cv + r * s;
    int w = 0;
    for (int p = 0; p < s; ++p) {
      if (a[p] < 0) continue;
      int better_cnt = 0;
      for (int q = 0; q < s; ++q) {
        if (q == p || a[q] < 0) continue;
        if (b[q] > b[p] || (b[q] == b[p] && a[q] < a[p])) ++better_cnt;
      }
      if (better_cnt < K) { co[r * K + w] = a[p]; cvo[r * K + w] = b[p]; ++w; }
    }
    for (; w < K; ++w) { co[r * K + w] = -1; cvo[r * K + w] = 0.0f; }
  }
}

template <int VPL>
cudaError_t launch_vpl(const float* acc, const float* comp, int64_t n, int C, int64_t ld, int K, int32_t* idx,
                       float* val, float* entropy, cudaStream_t st) {
  int64_t blocks = (n + 7) / 8;
  if (blocks > num_sms() * 16) blocks = num_sms() * 16;
  topk_kernel<VPL><<<(int)blocks, 256, 0, st>>>(acc, comp, n, C, ld, K, idx, val, entropy);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_topk(const float* acc, const float* comp, int64_t n, int C, int K, int32_t* idx, float* val,
                        float* entropy, cudaStream_t st, int64_t ld) {
  if (n <= 0) return cudaSuccess;
  if (ld <= 0) ld = C;
  if (C <= 32) return launch_vpl<1>(acc, comp, n, C, ld, K, idx, val, entropy, st);
  if (C <= 64) return launch_vpl<2>(acc, comp, n, C, ld, K, idx, val, entropy, st);
  if (C <= 128) return launch_vpl<4>(acc, comp, n, C, ld, K, idx, val, entropy, st);
  if (C <= 256) return launch_vpl<8>(acc, comp, n, C, ld, K, idx, val, entropy, st);
  if (C <= 512) return launch_vpl<16>(acc, comp, n, C, ld, K, idx, val, entropy, st);
  return launch_vpl<32>(acc, comp, n, C, ld, K, idx, val, entropy, st);
}

cudaError_t launch_code_topk(const int32_t* ci, const float* cv, int64_t R, int s, int K,
                             int32_t* ci_out, float* cv_out, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  int64_t blocks = (R + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  code_topk_kernel<<<(int)blocks, 256, 0, st>>>(ci, cv, R, s, K, ci_out, cv_out);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
