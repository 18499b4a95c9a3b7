// sgemm.cu -- FP32 SIMT (FFMA) GEMM: the full-precision comparison form of
// the codebook decode (Sec. 4.3, Eq. 8) and of the text similarity, against
// which the BF16 tensor-core path is measured.
//
//   out[M, N] = A[M, K] * B           B stored [K, N] (codebook) or, with
//                                     kBT, [N, K] (text vectors)
//   cosine epilogue: out / (|row| |column|), 0 where |row| < 1e-12 or |column| = 0
//
// 128 x 128 output tile per CTA of 256 threads, 8 x 8 accumulators per
// thread (rows ty + 16 i, columns tx + 16 j), K staged 8 at a time through
// shared memory.  All accumulation is FP32.
#include "scoup_internal.cuh"

namespace scoup {
namespace {

constexpr int SBM = 128, SBN = 128, SBK = 8;

template <bool kBT>
__global__ void __launch_bounds__(256) sgemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                    float* __restrict__ out, int64_t M, int N, int K,
                                                    const float* __restrict__ rownorm2,
                                                    const float* __restrict__ colnorm2) {
  __shared__ float As[SBK][SBM + 4];
  __shared__ float Bs[SBK][SBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * SBM;
  const int n0 = blockIdx.y * SBN;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  for (int k0 = 0; k0 < K; k0 += SBK) {
    for (int i = tid; i < SBM * SBK; i += 256) {
      const int r = i / SBK, c = i % SBK;
      const int64_t gr = m0 + r;
      As[c][r] = (gr < M && k0 + c < K) ? A[gr * K + k0 + c] : 0.0f;
    }
    for (int i = tid; i < SBN * SBK; i += 256) {
      int c, nn;
      if (kBT) { nn = i / SBK; c = i % SBK; } else { c = i / SBN; nn = i % SBN; }
      const int gn = n0 + nn, gk = k0 + c;
      float v = 0.0f;
      if (gn < N && gk < K) v = kBT ? B[(int64_t)gn * K + gk] : B[(int64_t)gk * N + gn];
      Bs[c][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + ty + 16 * i;
    if (r >= M) continue;
    float rinv = 1.0f;
    if (rownorm2) {
      const float rn = sqrtf(rownorm2[r]);
      rinv = rn < 1e-12f ? 0.0f : 1.0f / rn;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = n0 + tx + 16 * j;
      if (c >= N) continue;
      float x = acc[i][j];
      if (rownorm2) {
        const float cn = sqrtf(colnorm2[c]);
        x = (rinv == 0.0f || cn == 0.0f) ? 0.0f : x * rinv / cn;
      }
      out[r * N + c] = x;
    }
  }
}

// squared norms of the rows of a float32 [R, D] matrix, one warp per row
__global__ void row_norm2_f32_kernel(const float* __restrict__ X, int64_t R, int D, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; r < R;
       r += (int64_t)gridDim.x * blockDim.x / 32) {
    float s = 0.0f;
    for (int d = lane; d < D; d += 32) s = fmaf(X[r * D + d], X[r * D + d], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[r] = s;
  }
}

}  // namespace

cudaError_t launch_sgemm(const float* A, const float* B, bool b_transposed, float* out, int64_t M, int N, int K,
                         const float* rownorm2, const float* colnorm2, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((unsigned)((M + SBM - 1) / SBM), (unsigned)((N + SBN - 1) / SBN));
  if (b_transposed)
    sgemm_kernel<true><<<grid, 256, 0, st>>>(A, B, out, M, N, K, rownorm2, colnorm2);
  else
    sgemm_kernel<false><<<grid, 256, 0, st>>>(A, B, out, M, N, K, rownorm2, colnorm2);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_row_norm2_f32(const float* X, int64_t R, int D, float* out, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  int64_t blocks = (R * 32 + 255) / 256;
  if (blocks > num_sms() * 16) blocks = num_sms() * 16;
  row_norm2_f32_kernel<<<(int)blocks, 256, 0, st>>>(X, R, D, out);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
