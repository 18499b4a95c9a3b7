// filter.cu -- entropy filter of the uplifted Gaussians and the relevancy
// score of text queries.
//
// Entropy filter (the entropy analysis of Top-K filtering): keep the `keep`
// Gaussians of lowest coefficient entropy, ties to the lower index.  Every
// Gaussian gets the unique 64-bit key (order-preserving bits of H_i) << 32 | i;
// the key of rank keep - 1 is found exactly by an 8-pass radix select (one
// 256-bin histogram per pass; the last CTA of each pass picks the digit and
// updates the selection state in the workspace, so nothing returns to the
// host), then one pass marks the kept rows and clears the Top-K rows of the
// others to (-1, 0).
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

// Radix-select state, in the caller's workspace (cleared before the first pass).
struct SelectState {
  unsigned long long prefix;  // digits chosen so far
  unsigned long long pmask;   // their bits
  long long rank;             // rank of the wanted key among the keys matching the prefix
  unsigned int done;          // CTAs finished in the current pass
  unsigned int pad;
  uint32_t hist[256];
};

// One pass: histogram of digit `shift` over the keys that match the prefix;
// the last CTA turns it into the next digit (the bin holding `rank`), clears
// the histogram and the CTA counter for the next pass.
__global__ void __launch_bounds__(256) select_pass_kernel(const float* __restrict__ H, int64_t n, int shift,
                                                          long long rank0, SelectState* __restrict__ st) {
  __shared__ uint32_t sh[256];
  __shared__ bool s_last;
  const unsigned long long prefix = st->prefix, pmask = st->pmask;
  for (int b = threadIdx.x; b < 256; b += blockDim.x) sh[b] = 0u;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = entropy_key(H[i], i);
    if ((k & pmask) == prefix) atomicAdd(&sh[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x)
    if (sh[b]) atomicAdd(&st->hist[b], sh[b]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    // bins 8 lane .. 8 lane + 7; inclusive scan of their sums across the warp
    const int lane = threadIdx.x;
    const long long rank = shift == 56 ? rank0 : st->rank;
    uint32_t c[8], sum = 0;
    for (int d = 0; d < 8; ++d) { c[d] = __ldcg(&st->hist[lane * 8 + d]); sum += c[d]; }
    unsigned long long incl = sum;
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const unsigned long long excl = incl - sum;
    if ((unsigned long long)rank >= excl && (unsigned long long)rank < incl) {
      unsigned long long cum = excl;
      for (int d = 0; d < 8; ++d) {
        if ((unsigned long long)rank < cum + c[d]) {
          st->prefix = prefix | ((unsigned long long)(lane * 8 + d) << shift);
          st->pmask = pmask | (0xffull << shift);
          st->rank = rank - (long long)cum;
          break;
        }
        cum += c[d];
      }
    }
    for (int d = 0; d < 8; ++d) st->hist[lane * 8 + d] = 0u;
    if (lane == 0) st->done = 0u;
  }
}

__global__ void filter_kernel(const float* __restrict__ H, int64_t n, const SelectState* __restrict__ sel,
                              int keep_all, int keep_none, int K, int32_t* __restrict__ idx,
                              float* __restrict__ val, uint8_t* __restrict__ mask) {
  const unsigned long long thr = keep_all ? ~0ull : sel->prefix;
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
        if (p0 + u < P && lane < nq) R[(p0 + u) * nq + lane] = relevancy_term(alpha, c, sq);
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
      R[p * nq + q] = relevancy_term(alpha, smax, sq);
    }
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > num_sms() * 8) b = num_sms() * 8;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

size_t entropy_filter_state_bytes() { return sizeof(SelectState); }

int entropy_filter_run(const float* H, int64_t n, int64_t keep, int K, int32_t* idx, float* val, uint8_t* mask,
                       void* workspace, cudaStream_t st) {
  cudaError_t e;
  SelectState* sel = reinterpret_cast<SelectState*>(workspace);
  const int keep_none = keep <= 0;
  const int keep_all = keep >= n;
  if (!keep_none && !keep_all) {
    if ((e = cudaMemsetAsync(sel, 0, sizeof(SelectState), st)) != cudaSuccess)
      return set_error(SCOUP_ERR_CUDA, cudaGetErrorString(e));
    for (int shift = 56; shift >= 0; shift -= 8) {
      select_pass_kernel<<<grid_for(n), 256, 0, st>>>(H, n, shift, (long long)(keep - 1), sel);
      g_launches += 1;
    }
  }
  filter_kernel<<<grid_for(n), 256, 0, st>>>(H, n, sel, keep_all, keep_none, K, idx, val, mask);
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
