// gemm.cu -- BF16 tensor-core GEMM on tcgen05 for the codebook decode
// (paper Sec. 4.3, Eq. 8: F = What C) and the text-query similarity.
//
//   out[M, N] = A[M, K] * Bt[N, K]^T      (A, Bt bf16, K-major; f32 accumulate)
//
// One CTA computes a BM x BN tile (BM = 128).  Warp 0 issues TMA loads of
// 128-byte-swizzled K-major A and Bt tiles (BK = 64 bf16 = one swizzle row)
// into a kStages-deep shared-memory ring guarded by mbarriers; warp 1
// allocates BN TMEM columns and one thread issues tcgen05.mma (M=128, N=BN,
// K=16, four per stage), releasing each stage with tcgen05.commit; warps 2-5
// read the f32 accumulator back with tcgen05.ld (each warp its 32-lane TMEM
// quarter, one output row per thread) and run the epilogue:
//   kOutBF16 : bf16 output, optional per-row sum of squares of the rounded values
//   kOutF32  : f32 output
//   kOutCos  : f32 output / (|row| |column|), 0 where |row| < 1e-12
// Every mbarrier wait is bounded; a wait that gives up records an error in
// *status and the CTA frees its TMEM and leaves.
#include <cuda.h>
#include <cuda_bf16.h>

#include "scoup_internal.cuh"
#include "sm100_ptx.cuh"

namespace scoup {


namespace {

constexpr int BM = 128, BK = 64;
constexpr int kStages = 2;
constexpr int kGemmThreads = 192;
constexpr uint32_t kWaitIters = 1u << 22;

template <int BN>
struct GemmSmem {
  alignas(1024) __nv_bfloat16 a[kStages][BM * BK];
  alignas(1024) __nv_bfloat16 b[kStages][BN * BK];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t done;
  uint32_t tmem;
  int abort;
};

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                    const __grid_constant__ CUtensorMap tmB,
                                                                    GemmEpi ep) {
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  // align the carve-up to 1024 bytes (swizzle atoms)
  unsigned char* base = gsm_raw + ((1024 - (ptx::smem_u32(gsm_raw) & 1023u)) & 1023u);
  GemmSmem<BN>& sm = *reinterpret_cast<GemmSmem<BN>*>(base);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kt = (ep.K + BK - 1) / BK;
  constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
  constexpr uint32_t kBytesA = BM * BK * 2, kBytesB = BN * BK * 2;
  constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&sm.full[s], 1);
      ptx::mbar_init(&sm.empty[s], 1);
    }
    ptx::mbar_init(&sm.done, 1);
    sm.abort = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tmA);
    ptx::prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    ptx::tmem_alloc(&sm.tmem, kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = sm.tmem;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    for (int kb = 0; kb < kt; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages && !ptx::mbar_wait_bounded(&sm.empty[s], ((kb / kStages) - 1) & 1, kWaitIters)) {
        atomicOr(ep.status, kStatTimeout);
        sm.abort = 1;
        break;
      }
      ptx::mbar_arrive_expect_tx(&sm.full[s], kBytesA + kBytesB);
      ptx::tma_load_2d(sm.a[s], &tmA, &sm.full[s], kb * BK, m0);
      ptx::tma_load_2d(sm.b[s], &tmB, &sm.full[s], kb * BK, n0);
    }
    // wait (bounded) for the last copy issued into each stage before leaving
    for (int s = 0; s < kStages && s < kt; ++s) {
      const int kb_last = s + ((kt - 1 - s) / kStages) * kStages;
      if (!ptx::mbar_wait_bounded(&sm.full[s], (kb_last / kStages) & 1, kWaitIters)) atomicOr(ep.status, kStatTimeout);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    bool ok = true;
    for (int kb = 0; kb < kt && ok; ++kb) {
      const int s = kb % kStages;
      if (!ptx::mbar_wait_bounded(&sm.full[s], (kb / kStages) & 1, kWaitIters)) {
        atomicOr(ep.status, kStatTimeout);
        ok = false;
        break;
      }
      ptx::tc_fence_after();
      const uint32_t sa = ptx::smem_u32(sm.a[s]), sb = ptx::smem_u32(sm.b[s]);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        const uint64_t da = ptx::smem_desc_k128(sa + k * 32);
        const uint64_t db = ptx::smem_desc_k128(sb + k * 32);
        ptx::mma_f16(tmem, da, db, idesc, (kb > 0 || k > 0) ? 1u : 0u);
      }
      ptx::mma_commit(&sm.empty[s]);
    }
    ptx::mma_commit(&sm.done);  // arrives once every issued MMA has completed
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = m0 + q * 32 + lane;
    const bool waited = ptx::mbar_wait_bounded(&sm.done, 0, kWaitIters);
    ptx::tc_fence_after();
    if (!waited) {
      if (lane == 0) atomicOr(ep.status, kStatTimeout);
    } else {
      float ss = 0.0f;
      float rinv = 0.0f;
      if (ep.mode == kOutCos && row < ep.M) {
        const float rn = sqrtf(ep.rownorm2[row]);
        rinv = rn < 1e-12f ? 0.0f : 1.0f / rn;
      }
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        ptx::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (row >= ep.M) continue;
        const int col0 = n0 + c0;
        if (ep.mode == kOutBF16) {
          __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(ep.out) + (int64_t)row * ep.ldo + col0;
#pragma unroll
          for (int i = 0; i < 32; i += 2) {
            if (col0 + i + 1 < ep.N) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(v[i], v[i + 1]);
              *reinterpret_cast<__nv_bfloat162*>(o + i) = h;
              const float2 f = __bfloat1622float2(h);
              ss += f.x * f.x + f.y * f.y;
            } else if (col0 + i < ep.N) {
              const __nv_bfloat16 h = __float2bfloat16_rn(v[i]);
              o[i] = h;
              const float f = __bfloat162float(h);
              ss += f * f;
            }
          }
        } else {
          float* o = reinterpret_cast<float*>(ep.out) + (int64_t)row * ep.ldo + col0;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if (col0 + i < ep.N) {
              float x = v[i];
              if (ep.mode == kOutCos) {
                const float cn = ep.colnorm[col0 + i];
                x = (rinv == 0.0f || cn == 0.0f) ? 0.0f : x * rinv / cn;
              }
              o[i] = x;
            }
          }
        }
      }
      if (ep.mode == kOutBF16 && ep.rownorm2 && row < ep.M) atomicAdd(&ep.rownorm2[row], ss);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// K-major bf16 matrix [rows, K] (row stride K elements), box [box_rows, 64], 128-byte swizzle.
bool make_tmap(CUtensorMap* m, const void* ptr, int64_t rows, int K, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_bn(const void* A, const void* Bt, const GemmEpi& ep, cudaStream_t st) {
  CUtensorMap ta, tb;
  if (!make_tmap(&ta, A, ep.M, ep.K, BM) || !make_tmap(&tb, Bt, ep.N, ep.K, BN)) return cudaErrorInvalidValue;
  const size_t smem = sizeof(GemmSmem<BN>) + 1024;
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((ep.M + BM - 1) / BM), (unsigned)((ep.N + BN - 1) / BN));
  gemm_bf16_kernel<BN><<<grid, kGemmThreads, smem, st>>>(ta, tb, ep);
  g_launches += 1;
  return cudaGetLastError();
}

// ---- small conversion kernels ----
__global__ void f32_to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; i < n; i += (int64_t)gridDim.x * blockDim.x * 4) {
    if (i + 3 < n) {
      const float4 v = *reinterpret_cast<const float4*>(x + i);
      *reinterpret_cast<__nv_bfloat162*>(y + i) = __floats2bfloat162_rn(v.x, v.y);
      *reinterpret_cast<__nv_bfloat162*>(y + i + 2) = __floats2bfloat162_rn(v.z, v.w);
    } else {
      for (int64_t j = i; j < n; ++j) y[j] = __float2bfloat16_rn(x[j]);
    }
  }
}

// Bt[d][c] = bf16(B[c][d])  (B is [Cdim, D] row-major)
__global__ void transpose_bf16_kernel(const float* __restrict__ B, __nv_bfloat16* __restrict__ Bt, int Cdim, int D) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)Cdim * D;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / Cdim), c = (int)(i % Cdim);
    Bt[i] = __float2bfloat16_rn(B[(int64_t)c * D + d]);
  }
}

// norms (or squared norms) of the rows of a bf16 [R, D] matrix
__global__ void row_norm_bf16_kernel(const __nv_bfloat16* __restrict__ X, int64_t R, int D, float* __restrict__ out,
                                     int squared) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; r < R;
       r += (int64_t)gridDim.x * blockDim.x / 32) {
    float s = 0.0f;
    for (int d = lane; d < D; d += 32) {
      const float v = __bfloat162float(X[r * D + d]);
      s += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[r] = squared ? s : sqrtf(s);
  }
}

int blocks_for(int64_t n, int per) {
  int64_t b = (n + per - 1) / per;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_gemm_bf16(const void* A, const void* Bt, const GemmEpi& ep, cudaStream_t st) {
  if (ep.M <= 0 || ep.N <= 0) return cudaSuccess;
  if (ep.N <= 32) return launch_bn<32>(A, Bt, ep, st);
  if (ep.N <= 64) return launch_bn<64>(A, Bt, ep, st);
  if (ep.N <= 128) return launch_bn<128>(A, Bt, ep, st);
  return launch_bn<256>(A, Bt, ep, st);
}

cudaError_t launch_f32_to_bf16(const float* x, void* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  f32_to_bf16_kernel<<<blocks_for(n / 4 + 1, 256), 256, 0, st>>>(x, (__nv_bfloat16*)y, n);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const float* B, void* Bt, int Cdim, int D, cudaStream_t st) {
  transpose_bf16_kernel<<<blocks_for((int64_t)Cdim * D, 256), 256, 0, st>>>(B, (__nv_bfloat16*)Bt, Cdim, D);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_row_norm_bf16(const void* X, int64_t R, int D, float* out, int squared, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  row_norm_bf16_kernel<<<blocks_for(R * 32, 256), 256, 0, st>>>((const __nv_bfloat16*)X, R, D, out, squared);
  g_launches += 1;
  return cudaGetLastError();
}

bool gemm_tma_available() { return encode_fn() != nullptr; }

}  // namespace scoup
