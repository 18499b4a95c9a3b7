// render_mma.cu -- sparse coefficient rendering (Sec. 4.3, Eq. 7) as a
// tensor-core contraction.
//
// For one 16x16 tile, What(p) = sum_i e_i(p) w^_i over the tile's
// front-to-back list.  Cut the list into chunks of 32 Gaussians: the weights
// of a chunk form a 256 x 32 matrix E (pixels x Gaussians, e_i(p) or 0) and
// its K-sparse codes a dense 32 x C matrix W, so the tile's code rows are
// the sum over chunks of E W.  The kernel keeps that sum in tensor memory
// (two 128-pixel halves x C FP32 columns) and adds every chunk with
// tcgen05.mma; the rows leave the SM once, at the end of the tile.
//
// One CTA per tile: 256 walkers (one thread per pixel) and a ninth warp that
// issues the MMAs.  The walkers order the list window by window as in the
// uplift (tile_order.cuh, on a named barrier of their own).  Per chunk every
// walker walks its pixel front to back over the chunk's Gaussians (the
// binary32 exponent, alpha test and T-stop rule of the uplift) and writes its
// row of E, the walkers expand the chunk's codes into W and arrive on the
// chunk buffer's mbarrier; the MMA warp waits on it, issues the chunk's MMAs
// and commits them to the buffer's completion barrier (every chunk, also one
// without MMAs, so the walkers are never two chunks ahead on a buffer).  The bf16 operands are split, e = e_hi +
// e_lo and w = w_hi + w_lo (each part rounded to bf16), and three MMAs add
// E_hi W_hi + E_hi W_lo + E_lo W_hi.  With u = 2^-8 (bf16 unit roundoff)
// each split leaves u^2 of its value and the dropped E_lo W_lo is below u^2
// of the product: at most about 3 u^2 = 3 * 2^-16 (4.6e-5) relative per
// product before FP32 accumulation.
// Chunk buffers are double-buffered, so the walk of one chunk overlaps the
// MMAs of the previous one.  A chunk in which a pixel half has no weight
// issues no MMA for that half.
//
// Every wait (the MMA warp's on a chunk, the walkers' on a completion) is
// bounded; a wait that gives up sets the timeout status, the walkers stop,
// a stop still reaches the MMA warp, and TMEM is freed on every path.  The
// tile's rows are written at the end through the free chunk buffers, in
// coalesced 512-byte pieces.
#include <cuda_bf16.h>
#include <math.h>

#include "sm100_ptx.cuh"
#include "tile_order.cuh"

namespace scoup {
namespace {

constexpr int kMThreads = 256;  // walkers: one thread per pixel of the 16 x 16 tile
constexpr int kMWarps = kMThreads / 32;
constexpr int kMmaWarp = kMWarps;               // a ninth warp issues the tensor-core MMAs
constexpr int kCtaThreads = kMThreads + 32;
constexpr int kChunk = 32;      // Gaussians per chunk (contraction depth of one round of MMAs)
constexpr int kMaxN = 256;      // widest code row: two 128-lane halves of N FP32 TMEM columns
constexpr int kMaxK = 16;       // largest Top-K staged per window
constexpr uint32_t kWaitIters = 1u << 22;
using MOrder = OrderSmem<256, 10, kMThreads>;  // the walkers order alone (named barrier 1)

// Operand tiles are K-major without swizzle, built from 8-row x 16-byte core
// matrices: the 4 core matrices of an 8-row group (32 bf16 along K) are
// adjacent (LBO = 128 bytes) and the 8-row groups follow each other (SBO =
// 512 bytes).  A K = 16 slice starts 2 core matrices (256 bytes) further.
constexpr uint32_t kLBO = 128, kSBO = 512;
constexpr int kEBytes = 128 * kChunk * 2;    // one 128-pixel E tile: 8 KB
constexpr int kWBytes = kMaxN * kChunk * 2;  // one W tile: 16 KB

__device__ __forceinline__ int core_off(int row, int k) {
  return (row >> 3) * (int)kSBO + (k >> 3) * (int)kLBO + (row & 7) * 16 + (k & 7) * 2;
}

struct alignas(128) ChunkBuf {
  unsigned char e[2][2][kEBytes];  // [hi, lo][pixel half]
  unsigned char w[2][kWBytes];     // [hi, lo]
};

struct RenderMmaSmem {
  ChunkBuf buf[2];
  MOrder ord;
  float4 rec_a[MOrder::kWin];
  float4 rec_b[MOrder::kWin];
  float code_val[kMaxK * MOrder::kWin];  // entry-major: [k][window position]
  short code_idx[kMaxK * MOrder::kWin];
  uint64_t mma_done[2];  // per chunk buffer: the MMAs that read it have completed
  uint64_t ready[2];     // per chunk buffer: the walkers have written E and W (and ctl)
  uint64_t fin;
  uint32_t tmem;
  int any_e[kMWarps];
  int ctl[2][3];  // per chunk buffer: MMAs for pixel half 0, half 1; stop
  unsigned long long cnt[2];
};

static_assert(sizeof(ChunkBuf) * 2 >= kMWarps * 16384, "the epilogue stages 16 KB per warp in the chunk buffers");

// TMEM columns: a power of two holding two halves of Np columns, each half a
// multiple of 32 columns (the width of one tcgen05.ld).
__host__ __device__ inline uint32_t mma_tmem_cols(int Np) {
  uint32_t c = 64;
  while (c < 2u * (uint32_t)Np) c <<= 1;
  return c;
}

__device__ __forceinline__ void split_bf16x2(float x, float y, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Walks the thread's pixel over window positions j0 .. j0 + 31 and writes its
// row of E (hi and lo parts, zero where a Gaussian does not contribute);
// returns whether any weight of the row is nonzero.
// Gaussians that cannot pass the alpha test at any pixel of the warp's 16 x 2
// block (box_may_hit) are skipped, 8 at a time when none of 8 can.
__device__ __forceinline__ bool walk_chunk(const RenderMmaSmem& sm, int j0, int m, int wbase, float fpx, float fpy,
                                           float bx0, float by0, float& T, int& last, bool& done, unsigned& n_eval,
                                           unsigned& n_contrib, unsigned char* e_hi, unsigned char* e_lo, int row) {
  unsigned rel = 0u;
  if (!__all_sync(0xffffffffu, done)) {
    const int jl = j0 + (int)(threadIdx.x & 31);
    bool r = false;
    if (jl < m) {
      ProjRec pr;
      pr.a = sm.rec_a[jl];
      pr.b = sm.rec_b[jl];
      r = box_may_hit(pr, bx0, by0, (float)kTile, 2.0f);
    }
    rel = __ballot_sync(0xffffffffu, r);
  }
  bool any = false;
#pragma unroll
  for (int g = 0; g < kChunk / 8; ++g) {
    const unsigned rel8 = (rel >> (8 * g)) & 0xffu;
    if (rel8 == 0u) {  // warp-uniform
      *reinterpret_cast<uint4*>(e_hi + core_off(row, g * 8)) = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(e_lo + core_off(row, g * 8)) = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    // independent per Gaussian: exponent, alpha test and alpha (8 chains in
    // flight).  Positions past the window hold records that never pass (tau =
    // +inf), and a Gaussian outside the warp's box cannot pass either, so
    // alpha > 0 exactly when the Gaussian passes the alpha test here.
    float al[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + g * 8 + u;
      const float4 a = sm.rec_a[j];
      const float4 b = sm.rec_b[j];
      const float dx = a.x - fpx, dy = a.y - fpy;
      const float power = fmaf(dx, fmaf(a.z, dx, __fmul_rn(a.w, dy)), __fmul_rn(__fmul_rn(b.x, dy), dy));
      al[u] = (power <= 0.0f && power >= b.z) ? fminf(0.99f, b.y * __expf(power)) : 0.0f;
    }
    // serial front to back: transmittance, T-stop, weights
    float ev[8];
    const bool open0 = !done;
    int ustop = 8;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float test = T * (1.0f - al[u]);
      const bool act = !done && al[u] > 0.0f;
      const bool stop = act && test < 1e-4f;
      const bool tk = act && !stop;
      ev[u] = tk ? al[u] * T : 0.0f;
      T = tk ? test : T;
      if (tk) last = wbase + j0 + g * 8 + u + 1;
      n_contrib += tk ? 1u : 0u;
      if (stop) ustop = u;
      done = done || stop;
    }
    // examined: the group's Gaussians in the warp's box while the pixel was open, up to the stop
    if (open0) n_eval += __popc(rel8 & ((2u << ustop) - 1u));
    uint4 hi, lo;
    split_bf16x2(ev[0], ev[1], hi.x, lo.x);
    split_bf16x2(ev[2], ev[3], hi.y, lo.y);
    split_bf16x2(ev[4], ev[5], hi.z, lo.z);
    split_bf16x2(ev[6], ev[7], hi.w, lo.w);
    any = any || ((hi.x | hi.y | hi.z | hi.w) != 0u);
    *reinterpret_cast<uint4*>(e_hi + core_off(row, g * 8)) = hi;
    *reinterpret_cast<uint4*>(e_lo + core_off(row, g * 8)) = lo;
  }
  return any;
}

__device__ __forceinline__ uint32_t pack2_bf16(float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 32 columns c0 .. c0 + 31 of the pixel's row (fewer at the end of the row).
__device__ __forceinline__ void store_cols(void* __restrict__ out, int64_t pix, int C, int c0, bool bf16,
                                           const float (&v)[32]) {
  const int nc = min(32, C - c0);
  if (bf16) {
    __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out) + pix * C + c0;
    if (nc == 32 && (C & 7) == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        reinterpret_cast<uint4*>(o)[q] = make_uint4(pack2_bf16(v[8 * q], v[8 * q + 1]), pack2_bf16(v[8 * q + 2], v[8 * q + 3]),
                                                    pack2_bf16(v[8 * q + 4], v[8 * q + 5]),
                                                    pack2_bf16(v[8 * q + 6], v[8 * q + 7]));
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < nc) o[i] = __float2bfloat16_rn(v[i]);
    }
  } else {
    float* o = reinterpret_cast<float*>(out) + pix * C + c0;
    if (nc == 32 && (C & 3) == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        reinterpret_cast<float4*>(o)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < nc) o[i] = v[i];
    }
  }
}

// Barriers of the 256 walkers (named barrier 1; the MMA warp is not in it).
__device__ __forceinline__ void walkers_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool walkers_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, 1, 256, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0u;
}

// One CTA per tile; one CTA per SM (the accumulator takes the SM's 512 TMEM
// columns at C = 256, and the shared memory keeps a second CTA out).
__global__ void __launch_bounds__(kCtaThreads, 1) render_mma_kernel(
    CamArgs cam, const ProjRec* __restrict__ proj, const unsigned long long* __restrict__ keys,
    const uint32_t* __restrict__ tile_start, int slot, const int32_t* __restrict__ topk_idx,
    const float* __restrict__ topk_val, int K, int C, void* __restrict__ out, int out_bf16,
    float* __restrict__ out_T, int32_t* __restrict__ out_last, WsHeader* __restrict__ hdr) {
  extern __shared__ __align__(128) unsigned char msm_raw[];
  unsigned char* base = msm_raw + ((128u - (ptx::smem_u32(msm_raw) & 127u)) & 127u);
  RenderMmaSmem& sm = *reinterpret_cast<RenderMmaSmem*>(base);
  if (hdr->status & kStatCapacity) return;  // set by the binning before this launch: uniform
  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tile % cam.gx, ty = tile / cam.gx;
  const uint32_t begin = tile_start[tile];
  const int n = (int)(tile_start[tile + 1] - begin);
  const unsigned long long* tkeys = keys + begin;
  const int Np = (C + 15) & ~15;  // MMA N: C rounded up to a multiple of 16
  const uint32_t cols = mma_tmem_cols(Np), half_cols = cols / 2;

  if (tid == 0) {
    ptx::mbar_init(&sm.mma_done[0], 1);
    ptx::mbar_init(&sm.mma_done[1], 1);
    ptx::mbar_init(&sm.ready[0], kMThreads);
    ptx::mbar_init(&sm.ready[1], kMThreads);
    ptx::mbar_init(&sm.fin, 1);
    ptx::fence_mbar_init();
    sm.cnt[0] = sm.cnt[1] = 0ull;
  }
  if (warp == 0) {
    ptx::tmem_alloc(&sm.tmem, cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();  // the whole CTA: TMEM address and mbarriers are visible
  ptx::tc_fence_after();
  const uint32_t tmem = sm.tmem;

  if (warp == kMmaWarp) {
    // ---- MMA warp: one thread issues each chunk's MMAs once the walkers
    // have written it, and commits every chunk (also one without MMAs) to its
    // buffer's mma_done, so the walkers never run two chunks ahead of it ----
    if (lane == 0) {
      const uint32_t idesc = ptx::idesc_bf16_f32(128, Np);
      unsigned acc_init = 0u;  // bit h: pixel half h has received an MMA
      for (int chunk = 0;; ++chunk) {
        const int b = chunk & 1;
        if (!ptx::mbar_wait_bounded(&sm.ready[b], (uint32_t)(chunk >> 1) & 1u, kWaitIters)) {
          atomicOr(&hdr->status, kStatTimeout);
          break;
        }
        const int any0 = *(volatile int*)&sm.ctl[b][0], any1 = *(volatile int*)&sm.ctl[b][1];
        const int stop = *(volatile int*)&sm.ctl[b][2];
        if (stop) break;
        ptx::tc_fence_after();
        const ChunkBuf& cb = sm.buf[b];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!(h ? any1 : any0)) continue;
          const uint32_t d = tmem + (uint32_t)h * half_cols;
#pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint32_t ea = ptx::smem_u32(cb.e[pass == 2 ? 1 : 0][h]);
            const uint32_t wb = ptx::smem_u32(cb.w[pass == 1 ? 1 : 0]);
#pragma unroll
            for (int ks = 0; ks < kChunk / 16; ++ks)
              ptx::mma_f16(d, ptx::smem_desc_kmajor_none(ea + ks * 2 * kLBO, kLBO, kSBO),
                           ptx::smem_desc_kmajor_none(wb + ks * 2 * kLBO, kLBO, kSBO), idesc,
                           (((acc_init >> h) & 1u) || pass > 0 || ks > 0) ? 1u : 0u);
          }
        }
        acc_init |= (any0 ? 1u : 0u) | (any1 ? 2u : 0u);
        ptx::mma_commit(&sm.mma_done[b]);
      }
      // arrives once every MMA issued above has completed
      ptx::mma_commit(&sm.fin);
    }
    __syncwarp();
  } else {
  // ---- walkers ----
  const int px = tx * kTile + (tid & (kTile - 1)), py = ty * kTile + (tid >> 4);
  const bool inside = px < cam.width && py < cam.height;
  const int half = tid >> 7, row = tid & 127;  // E row and TMEM lane of this pixel
  float T = 1.0f;
  int last = 0;
  bool done = !inside;
  const OrderBuckets bk = order_buckets<MOrder>(hdr, slot);
  order_init<MOrder, 16>(sm.ord, tkeys, n, bk);

  unsigned n_eval = 0, n_contrib = 0;
  unsigned acc_init = 0u;  // bit h: pixel half h has received an MMA
  // thread 0: per chunk buffer b, bit b of `pending` = a chunk handed to the
  // MMA warp whose commit has not been waited for, bit b of `phase` = parity
  // of that commit's completion
  unsigned pending = 0u, phase = 0u;
  bool aborted = false, all_done = false;
  int chunk = 0, wbase = 0;
  OrderState ost;
  while (!all_done && !aborted) {
    const int m = n > 0 ? order_next_window<MOrder, 16>(sm.ord, tkeys, n, bk, ost, hdr) : 0;
    if (m <= 0) break;  // list exhausted, or an inconsistency (status already set)
    // records of the window; the positions up to the next chunk boundary get
    // a record no pixel accepts (tau = +inf)
    for (int j = tid; j < ((m + kChunk - 1) & ~(kChunk - 1)); j += kMThreads) {
      if (j < m) {
        const ProjRec pr = proj[(int)(sm.ord.win[j] & 0xffffffffull)];
        sm.rec_a[j] = pr.a;
        sm.rec_b[j] = pr.b;
      } else {
        sm.rec_a[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        sm.rec_b[j] = make_float4(0.0f, 0.0f, INFINITY, 0.0f);
      }
    }
    // one thread per Gaussian stages its whole code row (all loads in flight together)
    for (int j = tid; j < m; j += kMThreads) {
      const int64_t g = (int64_t)(sm.ord.win[j] & 0xffffffffull);
      int32_t ai[kMaxK];
      float av[kMaxK];
      if ((K & 3) == 0) {
#pragma unroll
        for (int k4 = 0; k4 < kMaxK / 4; ++k4)
          if (4 * k4 < K) {
            const int4 a = reinterpret_cast<const int4*>(topk_idx + g * K)[k4];
            const float4 v = reinterpret_cast<const float4*>(topk_val + g * K)[k4];
            ai[4 * k4] = a.x; ai[4 * k4 + 1] = a.y; ai[4 * k4 + 2] = a.z; ai[4 * k4 + 3] = a.w;
            av[4 * k4] = v.x; av[4 * k4 + 1] = v.y; av[4 * k4 + 2] = v.z; av[4 * k4 + 3] = v.w;
          }
      } else {
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
          if (k < K) {
            ai[k] = topk_idx[g * K + k];
            av[k] = topk_val[g * K + k];
          }
      }
#pragma unroll
      for (int k = 0; k < kMaxK; ++k)
        if (k < K) {
          sm.code_idx[k * MOrder::kWin + j] = (short)(ai[k] >= 0 && ai[k] < C ? ai[k] : -1);
          sm.code_val[k * MOrder::kWin + j] = av[k];
        }
    }
    walkers_sync();
    for (int j0 = 0; j0 < m; j0 += kChunk, ++chunk) {
      const int b = chunk & 1;
      ChunkBuf& cb = sm.buf[b];
      // the MMAs that last read this buffer have completed
      bool timed_out = false;
      if (tid == 0 && ((pending >> b) & 1u)) {
        timed_out = !ptx::mbar_wait_bounded(&sm.mma_done[b], (phase >> b) & 1u, kWaitIters);
        pending &= ~(1u << b);
        phase ^= 1u << b;
        if (timed_out) atomicOr(&hdr->status, kStatTimeout);
      }
      if (walkers_or(timed_out)) {
        aborted = true;
        break;
      }
      {
        const int n16 = Np * kChunk * 2 / 16;  // uint4 per W tile in use
        for (int i = tid; i < 2 * n16; i += kMThreads) {
          const int t = i >= n16 ? 1 : 0;
          reinterpret_cast<uint4*>(cb.w[t])[i - t * n16] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      const bool any = walk_chunk(sm, j0, m, wbase, (float)px, (float)py, (float)(tx * kTile),
                                  (float)(ty * kTile + 2 * warp), T, last, done, n_eval, n_contrib, cb.e[0][half],
                                  cb.e[1][half], row);
      const unsigned wany = __ballot_sync(0xffffffffu, any);
      if (lane == 0) sm.any_e[warp] = wany != 0u;
      walkers_sync();
      const bool any0 = (sm.any_e[0] | sm.any_e[1] | sm.any_e[2] | sm.any_e[3]) != 0;
      const bool any1 = (sm.any_e[4] | sm.any_e[5] | sm.any_e[6] | sm.any_e[7]) != 0;
      if (any0 || any1) {
        // W (hi, lo): entry (atom, Gaussian); repeated atoms of one code add up
        for (int t = tid; t < kChunk * K; t += kMThreads) {
          const int jc = t & (kChunk - 1), k = t >> 5;
          const int j = j0 + jc;
          if (j >= m) continue;
          const int atom = sm.code_idx[k * MOrder::kWin + j];
          if (atom < 0) continue;
          bool first = true;
          for (int k2 = 0; k2 < k; ++k2) first = first && sm.code_idx[k2 * MOrder::kWin + j] != atom;
          if (!first) continue;
          float v = sm.code_val[k * MOrder::kWin + j];
          for (int k2 = k + 1; k2 < K; ++k2)
            if (sm.code_idx[k2 * MOrder::kWin + j] == atom) v += sm.code_val[k2 * MOrder::kWin + j];
          const __nv_bfloat16 h = __float2bfloat16_rn(v);
          const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
          const int o = core_off(atom, jc);
          *reinterpret_cast<__nv_bfloat16*>(cb.w[0] + o) = h;
          *reinterpret_cast<__nv_bfloat16*>(cb.w[1] + o) = l;
        }
      }
      ptx::fence_async_shared();  // E and W are read by the tensor core (async proxy)
      const bool open = walkers_or(!done);
      // hand the chunk to the MMA warp (thread 0's control words are
      // published by its own arrival)
      if (tid == 0) {
        sm.ctl[b][0] = any0 ? 1 : 0;
        sm.ctl[b][1] = any1 ? 1 : 0;
        sm.ctl[b][2] = 0;
        pending |= 1u << b;
      }
      ptx::mbar_arrive(&sm.ready[b]);
      acc_init |= (any0 ? 1u : 0u) | (any1 ? 2u : 0u);
      if (!open) {
        all_done = true;
        ++chunk;  // the stop goes to the next chunk
        break;
      }
    }
    wbase += m;
  }

  // stop the MMA warp: the stop travels on the next chunk's buffer, once the
  // MMA warp has taken that buffer's previous chunk; then every MMA has
  // completed before the accumulator is read and TMEM freed
  bool fin_ok = true;
  {
    const int b = chunk & 1;
    if (tid == 0) {
      if ((pending >> b) & 1u) {
        fin_ok = ptx::mbar_wait_bounded(&sm.mma_done[b], (phase >> b) & 1u, kWaitIters);
        pending &= ~(1u << b);
        phase ^= 1u << b;
      }
      sm.ctl[b][2] = 1;
    }
    ptx::mbar_arrive(&sm.ready[b]);
  }
  if (tid == 0) {
    fin_ok = ptx::mbar_wait_bounded(&sm.fin, 0u, kWaitIters) && fin_ok;
    if (!fin_ok) atomicOr(&hdr->status, kStatTimeout);
  }
  const bool bad = walkers_or(!fin_ok) || aborted;
  ptx::tc_fence_after();

  // epilogue: each thread reads its own pixel's row (TMEM lane)
  const int q = warp & 3;
  const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)half * half_cols;
  const int64_t pix = (int64_t)py * cam.width + px;
  const bool have = ((acc_init >> half) & 1u) && !bad;  // uniform over the warp
  // Rows that split into 512-byte pieces (bf16 with C a multiple of 256, FP32
  // with C a multiple of 128) go through shared memory: the warp stages one
  // piece of each of its 32 pixel rows (16-byte chunks XOR-swizzled by row,
  // so neither the staging stores nor the reads conflict) in the chunk
  // buffers, free once the last MMA has completed, and writes every row's
  // piece with one coalesced warp store; other rows are stored per thread.
  const int esz = out_bf16 ? 2 : 4;
  const int piece_cols = 512 / esz;
  if (!bad && C == Np && C % piece_cols == 0 && ((uintptr_t)out & 15u) == 0) {
    unsigned char* stg = reinterpret_cast<unsigned char*>(&sm.buf[0]) + warp * 16384;
    unsigned char* orow = reinterpret_cast<unsigned char*>(out) + pix * (int64_t)C * esz;
    for (int p0 = 0; p0 < Np; p0 += piece_cols) {
      for (int c0 = p0; c0 < p0 + piece_cols; c0 += 32) {
        float v[32];
        if (have) {
          ptx::tmem_ld32(tb + (uint32_t)c0, v);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.0f;
        }
        const int k0 = (c0 - p0) * esz / 16;  // first 16-byte chunk of these columns in the piece
        if (out_bf16) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *reinterpret_cast<uint4*>(stg + lane * 512 + (((k0 + j) ^ lane) & 31) * 16) =
                make_uint4(pack2_bf16(v[8 * j], v[8 * j + 1]), pack2_bf16(v[8 * j + 2], v[8 * j + 3]),
                           pack2_bf16(v[8 * j + 4], v[8 * j + 5]), pack2_bf16(v[8 * j + 6], v[8 * j + 7]));
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<float4*>(stg + lane * 512 + (((k0 + j) ^ lane) & 31) * 16) =
                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
      __syncwarp();
      for (int r = 0; r < 32; ++r) {
        const uint4 val = *reinterpret_cast<const uint4*>(stg + r * 512 + ((lane ^ r) & 31) * 16);
        const unsigned long long ra = __shfl_sync(0xffffffffu, (unsigned long long)(uintptr_t)orow, r);
        if (__shfl_sync(0xffffffffu, inside, r))
          *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>((uintptr_t)ra) + p0 * esz + lane * 16) = val;
      }
      __syncwarp();
    }
  } else {
    for (int c0 = 0; c0 < Np; c0 += 32) {
      float v[32];
      if (have) {
        ptx::tmem_ld32(tb + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.0f;
      }
      if (inside && !bad) store_cols(out, pix, C, c0, out_bf16 != 0, v);
    }
  }
  if (inside) {
    if (out_T) out_T[pix] = T;
    if (out_last) out_last[pix] = last;
  }
  const unsigned we = __reduce_add_sync(0xffffffffu, n_eval);
  const unsigned wc = __reduce_add_sync(0xffffffffu, n_contrib);
  if (lane == 0) {
    atomicAdd(&sm.cnt[0], (unsigned long long)we);
    atomicAdd(&sm.cnt[1], (unsigned long long)wc);
  }
  }  // walkers
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) ptx::tmem_dealloc(tmem, cols);
  if (tid == 0) {
    atomicAdd(&hdr->evaluated, sm.cnt[0]);
    atomicAdd(&hdr->contributions, sm.cnt[1]);
  }
}

}  // namespace

bool render_mma_supported(int C, int K) { return C >= 1 && C <= kMaxN && K >= 1 && K <= kMaxK; }

size_t render_mma_smem_bytes() { return sizeof(RenderMmaSmem) + 128; }

cudaError_t launch_render_mma(const CamArgs& cam, const UpliftWs& ws, int slot, const int32_t* topk_idx,
                              const float* topk_val, int K, int C, void* out, int out_bf16, float* out_T,
                              int32_t* out_last, cudaStream_t st) {
  const int ntiles = cam.gx * cam.gy;
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = render_mma_smem_bytes();
  cudaError_t err = cudaFuncSetAttribute(render_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  render_mma_kernel<<<ntiles, kCtaThreads, smem, st>>>(cam, ws.proj, ws.keys, ws.tile_start, slot, topk_idx, topk_val,
                                                      K, C, out, out_bf16, out_T, out_last, ws.hdr);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
