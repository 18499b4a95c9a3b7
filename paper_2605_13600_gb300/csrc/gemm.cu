// gemm.cu -- BF16 tensor-core GEMM on tcgen05 for the codebook decode
// (paper Sec. 4.3, Eq. 8: F = What C) and the text-query similarity.
//
//   out[M, N] = A[M, K] * Bt[N, K]^T      (A, Bt bf16, K-major; f32 accumulate)
//
// Persistent: one CTA per SM walks the output in units of BM x BN (BM = 128).
// Warp 0 streams 128-byte-swizzled K-major A and Bt tiles (BK = 64 bf16, one
// swizzle row) with TMA into a kStages ring guarded by mbarriers; warp 1
// allocates two BN-column TMEM accumulators and one thread issues
// tcgen05.mma (M=128, N=BN, K=16) into them alternately, so the epilogue of
// one unit overlaps the MMAs of the next; warps 2-5 each own a 32-lane TMEM
// quarter (32 output rows), read 128-byte row chunks back with tcgen05.ld,
// apply the epilogue, stage them 128-byte-swizzled in shared memory and write
// them with TMA tile stores (double-buffered per warp).  Epilogues:
//   kOutBF16 : bf16 output, optional per-row sum of squares of the rounded values
//   kOutF32  : f32 output
//   kOutCos  : f32 output / (|row| |column|), 0 where |row| < 1e-12
// Every mbarrier wait is bounded; a wait that gives up records an error in
// *status, raises the CTA's abort flag, and every role leaves after draining
// its own copies in flight; TMEM is freed on every path.
#include <cuda.h>
#include <cuda_bf16.h>

#include "scoup_internal.cuh"
#include "sm100_ptx.cuh"

namespace scoup {
namespace {

constexpr int BM = 128, BK = 64;
constexpr int kGemmThreads = 192;
constexpr uint32_t kWaitIters = 1u << 22;

template <int BN>
struct GemmCfg {
  static constexpr int kStages = BN >= 256 ? 3 : 4;
  static constexpr uint32_t kTmemCols = 2 * BN;  // two accumulators
};

template <int BN>
struct GemmSmem {
  alignas(1024) __nv_bfloat16 a[GemmCfg<BN>::kStages][BM * BK];
  alignas(1024) __nv_bfloat16 b[GemmCfg<BN>::kStages][BN * BK];
  alignas(1024) unsigned char out[4][2][32 * 128];  // per epilogue warp, two 32-row x 128-byte chunks
  uint64_t full[GemmCfg<BN>::kStages];
  uint64_t empty[GemmCfg<BN>::kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem;
  volatile int abort;
};

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  if (ptx::mbar_wait_bounded(bar, parity, kWaitIters)) return true;
  atomicOr(status, kStatTimeout);
  *abort = 1;
  return false;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Position of a CTA's i-th unit.  Plain: units u = blockIdx.x + i gridDim.x
// in row-block-major order.  Fused query: the CTA's row blocks
// rb = blockIdx.x + j gridDim.x, each as its n_tiles column units followed by
// the query unit (so one epilogue thread sees every column of its row).
struct UnitPos {
  int m0, n0;
  bool query, valid;
};

template <int BN, bool kQuery>
__device__ __forceinline__ UnitPos unit_at(int i, int n_tiles, int m_blocks) {
  UnitPos p;
  if constexpr (!kQuery) {
    const int u = blockIdx.x + i * (int)gridDim.x;
    p.m0 = (u / n_tiles) * BM;
    p.n0 = (u % n_tiles) * BN;
    p.query = false;
    p.valid = u < m_blocks * n_tiles;
  } else {
    const int per = n_tiles + 1, rb = blockIdx.x + (i / per) * (int)gridDim.x, j = i % per;
    p.m0 = rb * BM;
    p.n0 = j * BN;
    p.query = j == n_tiles;
    p.valid = rb < m_blocks;
  }
  return p;
}

// kQuery: the fused query unit (compiled out of the plain launches).
template <int BN, bool kQuery>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                    const __grid_constant__ CUtensorMap tmB,
                                                                    const __grid_constant__ CUtensorMap tmO,
                                                                    const __grid_constant__ CUtensorMap tmG,
                                                                    const __grid_constant__ CUtensorMap tmS,
                                                                    GemmEpi ep) {
  using Cfg = GemmCfg<BN>;
  constexpr int kStages = Cfg::kStages;
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char* base = gsm_raw + ((1024 - (ptx::smem_u32(gsm_raw) & 1023u)) & 1023u);
  GemmSmem<BN>& sm = *reinterpret_cast<GemmSmem<BN>*>(base);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kt = (ep.K + BK - 1) / BK;
  const int n_tiles = (ep.N + BN - 1) / BN;
  const int m_blocks = (ep.M + BM - 1) / BM;
  constexpr bool fused = kQuery;
  constexpr uint32_t kBytesA = BM * BK * 2, kBytesB = BN * BK * 2;
  const uint32_t kBytesG = (uint32_t)ep.sim_n * BK * 2;
  constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);
  const uint32_t idesc_q = ep.sim_n == 16 ? ptx::idesc_bf16_f32(BM, 16) : ptx::idesc_bf16_f32(BM, 32);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&sm.full[s], 1);
      ptx::mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&sm.acc_full[b], 1);
      ptx::mbar_init(&sm.acc_empty[b], 4);
    }
    ptx::mbar_init(&sm.drain, 1);
    sm.abort = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tmA);
    ptx::prefetch_tmap(&tmB);
    ptx::prefetch_tmap(&tmO);
    if (fused) {
      ptx::prefetch_tmap(&tmG);
      ptx::prefetch_tmap(&tmS);
    }
  }
  if (warp == 1) {
    ptx::tmem_alloc(&sm.tmem, Cfg::kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = sm.tmem;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int it = 0;
    for (int i = 0; !sm.abort && !ep.stall_loads; ++i) {
      const UnitPos t = unit_at<BN, kQuery>(i, n_tiles, m_blocks);
      if (!t.valid) break;
      const CUtensorMap* mb = t.query ? &tmG : &tmB;
      const int nb = t.query ? 0 : t.n0;
      for (int kb = 0; kb < kt; ++kb, ++it) {
        const int s = it % kStages;
        if (it >= kStages && !wait_or_abort(&sm.empty[s], ((it / kStages) - 1) & 1, &sm.abort, ep.status)) break;
        ptx::mbar_arrive_expect_tx(&sm.full[s], kBytesA + (t.query ? kBytesG : kBytesB));
        ptx::tma_load_2d(sm.a[s], &tmA, &sm.full[s], kb * BK, t.m0);
        ptx::tma_load_2d(sm.b[s], mb, &sm.full[s], kb * BK, nb);
      }
    }
    // wait (bounded) for the last copy issued into each stage before leaving
    for (int s = 0; s < kStages && s < it; ++s) {
      const int last = s + ((it - 1 - s) / kStages) * kStages;
      if (!ptx::mbar_wait_bounded(&sm.full[s], (last / kStages) & 1, kWaitIters)) atomicOr(ep.status, kStatTimeout);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int it = 0, local = 0;
    bool ok = true;
    for (int i = 0; ok && !sm.abort; ++i, ++local) {
      const UnitPos t = unit_at<BN, kQuery>(i, n_tiles, m_blocks);
      if (!t.valid) break;
      const uint32_t id = t.query ? idesc_q : idesc;
      const int b = local & 1, use = local >> 1;
      if (local >= 2 && !wait_or_abort(&sm.acc_empty[b], (use - 1) & 1, &sm.abort, ep.status)) break;
      ptx::tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(b * BN);
      for (int kb = 0; kb < kt; ++kb, ++it) {
        const int s = it % kStages;
        if (!wait_or_abort(&sm.full[s], (it / kStages) & 1, &sm.abort, ep.status)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t sa = ptx::smem_u32(sm.a[s]), sb = ptx::smem_u32(sm.b[s]);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          ptx::mma_f16(d, ptx::smem_desc_k128(sa + k * 32), ptx::smem_desc_k128(sb + k * 32), id,
                       (kb > 0 || k > 0) ? 1u : 0u);
        ptx::mma_commit(&sm.empty[s]);
      }
      if (ok) ptx::mma_commit(&sm.acc_full[b]);
    }
    // every issued MMA has completed once `drain` flips
    ptx::mma_commit(&sm.drain);
    if (!ptx::mbar_wait_bounded(&sm.drain, 0, kWaitIters)) atomicOr(ep.status, kStatTimeout);
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    constexpr int kCW = 64;  // bf16 columns per 128-byte chunk (32 for f32 output)
    int local = 0, sbuf = 0;
    float ss_row = 0.0f;  // fused query: squared norm of the row's rounded outputs over its row block
    for (int i = 0; !sm.abort; ++i, ++local) {
      const UnitPos t = unit_at<BN, kQuery>(i, n_tiles, m_blocks);
      if (!t.valid) break;
      const int m0 = t.m0, n0 = t.query ? 0 : t.n0;
      const int mode = (kQuery && t.query) ? ep.sim_mode : ep.mode;
      const bool f32out = mode != kOutBF16;
      const int cw = f32out ? 32 : kCW;
      const int ncols = (kQuery && t.query) ? ep.sim_n : BN;  // accumulator columns of this unit (sim_n <= 32)
      const int nlim = t.query ? ep.sim_n : ep.N;
      const bool write = kQuery ? (t.query || ep.store) : true;
      const CUtensorMap* mo = t.query ? &tmS : &tmO;
      const int b = local & 1, use = local >> 1;
      if (!wait_or_abort(&sm.acc_full[b], use & 1, &sm.abort, ep.status)) break;
      ptx::tc_fence_after();
      const int row = m0 + q * 32 + lane;
      if (fused && !t.query && t.n0 == 0) ss_row = 0.0f;
      float rinv = 0.0f;
      if ((mode == kOutCos || mode == kOutRel) && row < ep.M) {
        const float rn = sqrtf(t.query ? ss_row : ep.rownorm2[row]);
        rinv = rn < 1e-12f ? 0.0f : 1.0f / rn;
      }
      float ss = 0.0f;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN);
      for (int c0 = 0; c0 < ncols; c0 += cw) {
        float v[kCW];
        ptx::tmem_ld32(tbase + (uint32_t)c0, *reinterpret_cast<float(*)[32]>(&v[0]));
        if (!f32out) ptx::tmem_ld32(tbase + (uint32_t)(c0 + 32), *reinterpret_cast<float(*)[32]>(&v[32]));
        if (c0 + cw >= ncols) {
          // the accumulator is drained: the MMA warp may reuse it
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&sm.acc_empty[b]);
        }
        // a box that starts past the last row or column stores nothing: skip it
        if (n0 + c0 >= nlim || m0 + q * 32 >= ep.M) continue;
        unsigned char* buf = sm.out[q][sbuf];
        if (write) {
          if (lane == 0) ptx::bulk_wait_read<1>();  // this buffer's previous store has read it
          __syncwarp();
        }
        unsigned char* rowp = buf + lane * 128;
        if (!f32out) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            uint4 w;
            w.x = pack_bf16x2(v[8 * j + 0], v[8 * j + 1]);
            w.y = pack_bf16x2(v[8 * j + 2], v[8 * j + 3]);
            w.z = pack_bf16x2(v[8 * j + 4], v[8 * j + 5]);
            w.w = pack_bf16x2(v[8 * j + 6], v[8 * j + 7]);
            if (write) *reinterpret_cast<uint4*>(rowp + ((j ^ (lane & 7)) << 4)) = w;
            if (ep.rownorm2 || fused) {
              const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
              for (int t2 = 0; t2 < 4; ++t2) {
                const float2 f = __bfloat1622float2(h[t2]);
                ss = fmaf(f.x, f.x, fmaf(f.y, f.y, ss));
              }
            }
          }
        } else {
          if (mode == kOutCos || mode == kOutRel) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int col = n0 + c0 + c;
              const float cn = col < nlim ? ep.colnorm[col] : 0.0f;
              v[c] = (rinv == 0.0f || cn == 0.0f) ? 0.0f : v[c] * rinv / cn;
            }
          }
          if (mode == kOutRel) {
            // Eq. 9 on the thread's whole row of similarities (at most 32
            // columns, one column tile): R_q = min_k 1 / (1 + e^{a (s_k - s_q)})
            // is the term of the largest canonical similarity; query q is
            // column n_canon + q, staged at column q of the relevancy row
            float smax = -INFINITY;
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (c < ep.n_canon) smax = fmaxf(smax, v[c]);
            float* rowf = reinterpret_cast<float*>(rowp);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int qq = c - ep.n_canon;
              if (qq >= 0 && c < nlim) {
                const float r = relevancy_term(ep.alpha, smax, v[c]);
                rowf[(((qq >> 2) ^ (lane & 7)) << 2) + (qq & 3)] = r;
              }
            }
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              *reinterpret_cast<float4*>(rowp + ((j ^ (lane & 7)) << 4)) =
                  make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          }
        }
        if (!write) continue;
        ptx::fence_async_shared();
        __syncwarp();
        if (lane == 0) {
          ptx::tma_store_2d(mo, buf, n0 + c0, m0 + q * 32);
          ptx::bulk_commit();
        }
        sbuf ^= 1;
      }
      if (fused) {
        if (!t.query) ss_row += ss;
        else if (ep.rownorm2 && row < ep.M) ep.rownorm2[row] = ss_row;
      } else if (!f32out && ep.rownorm2 && row < ep.M) {
        atomicAdd(&ep.rownorm2[row], ss);
      }
    }
    if (lane == 0) ptx::bulk_wait<0>();  // stores complete before the CTA leaves
    __syncwarp();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cfg::kTmemCols);
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

// Row-major 2-D matrix [rows, cols] (row stride cols elements), box
// [box_rows, box_cols], 128-byte swizzle (box_cols x element size = 128 bytes).
bool make_tmap(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize, int64_t rows, int64_t cols,
               int box_cols, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * (cuuint64_t)esize};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  return enc(m, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Gt (bf16 [sim_n, K]) is the fused query's operand; null without one.
template <int BN>
cudaError_t launch_bn(const void* A, const void* Bt, const void* Gt, const GemmEpi& ep, cudaStream_t st) {
  CUtensorMap ta, tb, to, tg, ts;
  const bool f32out = ep.mode != kOutBF16;
  const bool fused = ep.sim_n > 0;
  if (!make_tmap(&ta, A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ep.M, ep.K, BK, BM) ||
      !make_tmap(&tb, Bt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ep.N, ep.K, BK, BN))
    return cudaErrorInvalidValue;
  // without stored rows (fused query, store = 0) the output map is never used:
  // it is encoded on the operand Bt so that it is valid
  if (!ep.store) to = tb;
  else if (!(f32out ? make_tmap(&to, ep.out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ep.M, ep.ldo, 32, 32)
                    : make_tmap(&to, ep.out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ep.M, ep.ldo, 64, 32)))
    return cudaErrorInvalidValue;
  if (fused) {
    if (!make_tmap(&tg, Gt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ep.sim_n, ep.K, BK, ep.sim_n) ||
        !make_tmap(&ts, ep.sim_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ep.M, ep.sim_ldo, 32, 32))
      return cudaErrorInvalidValue;
  } else {
    tg = tb;  // unused
    ts = to;
  }
  const size_t smem = sizeof(GemmSmem<BN>) + 1024;
  auto kern = fused ? gemm_bf16_kernel<BN, true> : gemm_bf16_kernel<BN, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t m_blocks = (ep.M + BM - 1) / BM;
  const int64_t units = fused ? m_blocks : m_blocks * ((ep.N + BN - 1) / BN);
  const int grid = (int)(units < num_sms() ? units : num_sms());
  kern<<<grid, kGemmThreads, smem, st>>>(ta, tb, to, tg, ts, ep);
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
  if (b > num_sms() * 16) b = num_sms() * 16;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_gemm_bf16(const void* A, const void* Bt, const GemmEpi& ep, cudaStream_t st) {
  if (ep.M <= 0 || ep.N <= 0) return cudaSuccess;
  // bf16 output is read back from TMEM 64 columns at a time: BN >= 64 (the
  // columns past N are the zero fill of the Bt tile)
  if (ep.sim_n) return cudaErrorInvalidValue;  // launch_gemm_bf16_query
  if (ep.N <= 32 && ep.mode != kOutBF16) return launch_bn<32>(A, Bt, nullptr, ep, st);
  if (ep.N <= 64) return launch_bn<64>(A, Bt, nullptr, ep, st);
  if (ep.N <= 128) return launch_bn<128>(A, Bt, nullptr, ep, st);
  return launch_bn<256>(A, Bt, nullptr, ep, st);
}

cudaError_t launch_gemm_bf16_query(const void* A, const void* Bt, const void* Gt, const GemmEpi& ep,
                                   cudaStream_t st) {
  if (ep.M <= 0 || ep.N <= 0) return cudaSuccess;
  if (ep.mode != kOutBF16 || (ep.sim_n != 16 && ep.sim_n != 32) || !Gt || !ep.sim_out ||
      (ep.sim_mode != kOutCos && ep.sim_mode != kOutRel) || (ep.store && !ep.out))
    return cudaErrorInvalidValue;
  if (ep.N <= 64) return launch_bn<64>(A, Bt, Gt, ep, st);
  if (ep.N <= 128) return launch_bn<128>(A, Bt, Gt, ep, st);
  return launch_bn<256>(A, Bt, Gt, ep, st);
}

// One warp per (q, c): Gt[q][c] = bf16(sum_d text[q][d] codebook[c][d]) with
// FP32 sums; the warps of c = 0 also write |text_q|.
__global__ void text_codebook_kernel(const float* __restrict__ text, const float* __restrict__ codebook, int Q,
                                     int C, int D, __nv_bfloat16* __restrict__ Gt, float* __restrict__ tnorm) {
  const int lane = threadIdx.x & 31;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; w < (int64_t)Q * C;
       w += (int64_t)gridDim.x * blockDim.x / 32) {
    const int qi = (int)(w / C), c = (int)(w - (int64_t)qi * C);
    float dot = 0.0f, sq = 0.0f;
    for (int d = lane; d < D; d += 32) {
      const float t = text[(int64_t)qi * D + d];
      dot = fmaf(t, codebook[(int64_t)c * D + d], dot);
      sq = fmaf(t, t, sq);
    }
    for (int off = 16; off > 0; off >>= 1) {
      dot += __shfl_xor_sync(0xffffffffu, dot, off);
      sq += __shfl_xor_sync(0xffffffffu, sq, off);
    }
    if (lane == 0) {
      Gt[w] = __float2bfloat16_rn(dot);
      if (c == 0) tnorm[qi] = sqrtf(sq);
    }
  }
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

cudaError_t launch_text_codebook(const float* text, const float* codebook, int Q, int C, int D, void* Gt,
                                 float* tnorm, cudaStream_t st) {
  if (Q <= 0 || C <= 0) return cudaSuccess;
  text_codebook_kernel<<<blocks_for((int64_t)Q * C * 32, 256), 256, 0, st>>>(text, codebook, Q, C, D,
                                                                             (__nv_bfloat16*)Gt, tnorm);
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

// Runs a 128 x 64 x 64 GEMM whose producer issues no loads: the MMA and
// epilogue warps' bounded waits run out, the kernel records kStatTimeout and
// frees its TMEM, and the context stays usable.  Returns the device status.
int gemm_timeout_selftest(void* workspace, size_t ws_bytes, cudaStream_t st) {
  const size_t need = 256 + 3 * (size_t)128 * 64 * 2;
  if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255u)) return SCOUP_ERR_INVALID_ARG;
  char* w = (char*)workspace;
  int* status = (int*)w;
  void* A = w + 256;
  void* B = (char*)A + 128 * 64 * 2;
  void* out = (char*)B + 128 * 64 * 2;
  if (cudaMemsetAsync(w, 0, need, st) != cudaSuccess) return SCOUP_ERR_CUDA;
  GemmEpi ep;
  ep.M = 128;
  ep.N = 64;
  ep.K = 64;
  ep.mode = kOutBF16;
  ep.out = out;
  ep.ldo = 64;
  ep.rownorm2 = nullptr;
  ep.colnorm = nullptr;
  ep.status = status;
  ep.stall_loads = 1;
  if (launch_gemm_bf16(A, B, ep, st) != cudaSuccess) return SCOUP_ERR_CUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCOUP_ERR_CUDA;
  return (h & kStatTimeout) ? SCOUP_ERR_TIMEOUT : SCOUP_OK;
}

}  // namespace scoup
