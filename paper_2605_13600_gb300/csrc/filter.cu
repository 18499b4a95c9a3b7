// filter.cu -- entropy filter of the uplifted Gaussians and the relevancy
// score of text queries.
//
// Entropy filter (the entropy analysis of Top-K filtering): keep the `keep`
// Gaussians of lowest coefficient entropy, ties to the lower index.  Every
// Gaussian gets the unique 64-bit key (order-preserving bits of H_i) << 32 | i;
// the key of rank keep - 1 is found exactly by an 8-pass radix select (one
// 256-bin histogram per pass, the digit chosen on the host), then one pass
// marks the kept rows and clears the Top-K rows of the others to (-1, 0).
//
// Relevancy (App. B, Eq. 9): R = min_k e^{a s_q} / (e^{a s_q} + e^{a s_k})
// = min_k 1 / (1 + e^{a (s_k - s_q)}) from the similarity matrix, whose first
// n_canon columns are the canonical phrases and the rest the queries.
#include <math.h>

#include "scoup_internal.cuh"

namespace scoup {
namespace {

__device__ __forceinline__ unsigned long long entropy_key(float h, int64_t i) {
  uint32_t u = __float_as_uint(h);
  u ^= (u & 0x80000000u) ? 0xffffffffu : 0x80000000u;  // total order of the float values
  return ((unsigned long long)u << 32) | (uint32_t)i;
}

__global__ void key_hist_kernel(const float* __restrict__ H, int64_t n, unsigned long long prefix,
                                unsigned long long pmask, int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[256];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) sh[b] = 0u;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = entropy_key(H[i], i);
    if ((k & pmask) == prefix) atomicAdd(&sh[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

__global__ void filter_kernel(const float* __restrict__ H, int64_t n, unsigned long long thr, int keep_none,
                              int K, int32_t* __restrict__ idx, float* __restrict__ val,
                              uint8_t* __restrict__ mask) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool keep = !keep_none && entropy_key(H[i], i) <= thr;
    if (mask) mask[i] = keep ? 1 : 0;
    if (!keep && idx)
      for (int k = 0; k < K; ++k) {
        idx[i * K + k] = -1;
        val[i * K + k] = 0.0f;
      }
  }
}

// One warp per similarity row: lane q (and q + 32, ...) takes query q.
// 1 / (1 + e^{a (s_k - s_q)}) decreases in s_k (a > 0), so the minimum over
// the canonical phrases is the term of the largest canonical similarity:
// one exponential per output, the same value as the minimum of all terms.
// Rows of at most 32 columns are read four at a time, one coalesced word per
// lane and row (the loads of the four rows in flight together); the
// canonical maximum and each query's value come by shuffles.
constexpr int kRelRows = 4;

__global__ void relevancy_kernel(const float* __restrict__ sim, int64_t P, int ncols, int n_canon, float alpha,
                                 float* __restrict__ R) {
  const int nq = ncols - n_canon;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (ncols <= 32) {
    for (int64_t p0 = gw * kRelRows; p0 < P; p0 += warps * kRelRows) {
      float v[kRelRows];
#pragma unroll
      for (int u = 0; u < kRelRows; ++u)
        v[u] = (p0 + u < P && lane < ncols) ? sim[(p0 + u) * ncols + lane] : -INFINITY;
#pragma unroll
      for (int u = 0; u < kRelRows; ++u) {
        float c = lane < n_canon ? v[u] : -INFINITY;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, off));
        const float sq = __shfl_sync(0xffffffffu, v[u], min(n_canon + lane, 31));
        if (p0 + u < P && lane < nq) R[(p0 + u) * nq + lane] = fminf(1.0f, 1.0f / (1.0f + expf(alpha * (c - sq))));
      }
    }
    return;
  }
  for (int64_t p = gw; p < P; p += warps) {
    const float* row = sim + p * ncols;
    float smax = -INFINITY;
    for (int k = 0; k < n_canon; ++k) smax = fmaxf(smax, row[k]);
    for (int q = lane; q < nq; q += 32) {
      const float sq = row[n_canon + q];
      R[p * nq + q] = fminf(1.0f, 1.0f / (1.0f + expf(alpha * (smax - sq))));
    }
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > num_sms() * 8) b = num_sms() * 8;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

int entropy_filter_run(const float* H, int64_t n, int64_t keep, int K, int32_t* idx, float* val, uint8_t* mask,
                       uint32_t* hist, cudaStream_t st) {
  cudaError_t e;
  unsigned long long thr = ~0ull;
  const int keep_none = keep <= 0;
  if (keep > 0 && keep < n) {
    unsigned long long prefix = 0ull, pmask = 0ull;
    int64_t rank = keep - 1;
    for (int shift = 56; shift >= 0; shift -= 8) {
      if ((e = cudaMemsetAsync(hist, 0, 256 * sizeof(uint32_t), st)) != cudaSuccess) return set_error(SCOUP_ERR_CUDA, cudaGetErrorString(e));
      key_hist_kernel<<<grid_for(n), 256, 0, st>>>(H, n, prefix, pmask, shift, hist);
      g_launches += 1;
      uint32_t h[256];
      if ((e = cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return set_error(SCOUP_ERR_CUDA, cudaGetErrorString(e));
      int d = 0;
      while (d < 255 && rank >= (int64_t)h[d]) rank -= h[d++];
      prefix |= (unsigned long long)d << shift;
      pmask |= 0xffull << shift;
    }
    thr = prefix;
  }
  filter_kernel<<<grid_for(n), 256, 0, st>>>(H, n, thr, keep_none, K, idx, val, mask);
  g_launches += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return set_error(SCOUP_ERR_CUDA, cudaGetErrorString(e));
  return SCOUP_OK;
}

cudaError_t launch_relevancy(const float* sim, int64_t P, int ncols, int n_canon, float alpha, float* R,
                             cudaStream_t st) {
  if (P <= 0 || ncols <= n_canon) return cudaSuccess;
  relevancy_kernel<<<grid_for(P * 32), 256, 0, st>>>(sim, P, ncols, n_canon, alpha, R);  // a warp per row
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
