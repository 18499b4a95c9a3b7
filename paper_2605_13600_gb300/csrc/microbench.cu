// microbench.cu -- measurement helper: the GPU's FP32 atomic-update
// throughput to scattered addresses (the ceiling of the uplift's accumulator
// updates, one fire-and-forget reduction per (Gaussian, atom) update).
#include "scoup_internal.cuh"

namespace scoup {
namespace {

// A 32-bit mixing function of the update index (the finaliser of
// MurmurHash3): consecutive indices land on unrelated elements.
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__global__ void __launch_bounds__(256) red_kernel(float* __restrict__ buf, uint32_t mask, int64_t count,
                                                  uint32_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = mix32((uint32_t)i ^ mix32((uint32_t)(i >> 32) + seed)) & mask;
    atomicAdd(&buf[e], 1.0f);
  }
}

}  // namespace
}  // namespace scoup

extern "C" int scoup_selftest_red_throughput(float* buf, int32_t log2_n, int64_t count, uint32_t seed,
                                             void* stream) {
  if (!buf || log2_n < 10 || log2_n > 31 || count < 0)
    return scoup::set_error(SCOUP_ERR_INVALID_ARG, "scoup_selftest_red_throughput: buf, log2_n in [10, 31], count >= 0");
  if (count == 0) return SCOUP_OK;
  const uint32_t mask = (uint32_t)((1ull << log2_n) - 1ull);
  const int blocks = scoup::num_sms() * 8;
  scoup::red_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(buf, mask, count, seed);
  scoup::g_launches += 1;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCOUP_OK : scoup::set_error(SCOUP_ERR_CUDA, cudaGetErrorString(e));
}
