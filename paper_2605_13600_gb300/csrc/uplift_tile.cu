// uplift_tile.cu -- per-tile front-to-back compositing and sparse scatter
// (paper Sec. 3 Eq. 2; Sec. 4.2 Eq. 5; Algorithm 1).
//
// One CTA per 16x16 tile, one pixel per thread.  The tile's unordered key list
// (depth bits << 32 | Gaussian id) is consumed in windows of the kWin smallest
// remaining keys: a block-wide MSD radix select finds the window boundary, the
// window is gathered into shared memory and bitonic-sorted, and then composited
// in batches of 256 Gaussians staged in shared memory.  The tile stops as soon
// as every pixel has hit the transmittance cutoff, so the far part of a long
// list is never ordered.
//
// Scatter: codes are constant per region (Sec. 4.1), so for a Gaussian g the
// contributions of all pixels of one region r inside the tile can be summed
// first (distributivity) and flushed once as s atomics acc[g][j] += c_j * sum.
// Per Gaussian, each warp reduces its pixels' weights with shuffles when the
// warp lies in one region, and otherwise per lane; the per-(Gaussian, region)
// tile partials live in shared memory and are flushed after every batch.
#include <math.h>

#include "scoup_internal.cuh"

namespace scoup {
namespace {

constexpr int kThreads = 256;
constexpr int kWin = 1024;
constexpr int kMaxSlots = 8;
constexpr int kMaxS = 64;
constexpr unsigned kFull = 0xffffffffu;

struct TileSmem {
  unsigned long long win[kWin];
  float4 rec_a[kThreads];
  float4 rec_b[kThreads];
  int gid[kThreads];
  float part[kThreads][kMaxSlots];
  int slot_region[kMaxSlots];
  int slot_idx[kMaxSlots][kMaxS];
  float slot_val[kMaxSlots][kMaxS];
  int warp_regions[kThreads / 32][32];
  int warp_nreg[kThreads / 32];
  uint32_t hist[256];
  unsigned long long red_min, red_max;
  unsigned int cursor;
  int nslots;
  int sel_digit;
  int sel_rank;
  unsigned long long cnt[4];
};

__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Block-wide: the rank-th smallest key (0-based) among keys[i] with
// (first || keys[i] > last).  Keys are unique.  Requires rank < remaining.
__device__ unsigned long long select_rank(TileSmem& sm, const unsigned long long* __restrict__ keys,
                                          int n, unsigned long long last, bool first, int rank) {
  const int tid = threadIdx.x;
  if (tid == 0) { sm.red_min = ~0ull; sm.red_max = 0ull; }
  __syncthreads();
  unsigned long long lmin = ~0ull, lmax = 0ull;
  for (int i = tid; i < n; i += kThreads) {
    const unsigned long long k = keys[i];
    if (first || k > last) { lmin = min(lmin, k); lmax = max(lmax, k); }
  }
  for (int off = 16; off > 0; off >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(kFull, lmin, off));
    lmax = max(lmax, __shfl_xor_sync(kFull, lmax, off));
  }
  if ((tid & 31) == 0) { atomicMin(&sm.red_min, lmin); atomicMax(&sm.red_max, lmax); }
  __syncthreads();
  const unsigned long long base = sm.red_min, span = sm.red_max - sm.red_min;
  const int nbits = span ? 64 - __clzll((long long)span) : 1;
  unsigned long long prefix = 0ull, pmask = 0ull;
  for (int shift = ((nbits - 1) / 8) * 8; shift >= 0; shift -= 8) {
    sm.hist[tid] = 0u;
    __syncthreads();
    for (int i = tid; i < n; i += kThreads) {
      const unsigned long long k = keys[i];
      if (first || k > last) {
        const unsigned long long x = k - base;
        if ((x & pmask) == prefix) atomicAdd(&sm.hist[(x >> shift) & 255u], 1u);
      }
    }
    __syncthreads();
    if (tid < 32) {
      // each lane owns 8 consecutive digits
      uint32_t c[8], s = 0;
      for (int d = 0; d < 8; ++d) { c[d] = sm.hist[tid * 8 + d]; s += c[d]; }
      uint32_t incl = s;
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, incl, off);
        if (tid >= off) incl += y;
      }
      const uint32_t excl = incl - s;
      const bool mine = (uint32_t)rank >= excl && (uint32_t)rank < incl;
      if (mine) {
        uint32_t cum = excl;
        for (int d = 0; d < 8; ++d) {
          if ((uint32_t)rank < cum + c[d]) { sm.sel_digit = tid * 8 + d; sm.sel_rank = rank - (int)cum; break; }
          cum += c[d];
        }
      }
    }
    __syncthreads();
    prefix |= (unsigned long long)sm.sel_digit << shift;
    pmask |= 0xffull << shift;
    rank = sm.sel_rank;
    __syncthreads();
  }
  return base + prefix;
}

// Ascending bitonic sort of sm.win[0..P), P a power of two <= kWin.
__device__ void bitonic_sort(unsigned long long* win, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += kThreads) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = win[i], b = win[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { win[i] = b; win[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kThreads, 4) uplift_tile_kernel(
    CamArgs cam, const ProjRec* __restrict__ proj, const unsigned long long* __restrict__ keys,
    const uint32_t* __restrict__ tile_start, const int32_t* __restrict__ rmap, int32_t R_total,
    const int32_t* __restrict__ code_idx, const float* __restrict__ code_val, int s, int C,
    float* __restrict__ accum, WsHeader* __restrict__ hdr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(smem_raw);
  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t begin = tile_start[tile];
  const int n = (int)(tile_start[tile + 1] - begin);
  if (n == 0) return;
  if (hdr->status & kStatCapacity) return;
  const unsigned long long* tkeys = keys + begin;

  const int tx = tile % cam.gx, ty = tile / cam.gx;
  const int px = tx * kTile + (tid & (kTile - 1));
  const int py = ty * kTile + (tid >> 4);
  const bool inside = px < cam.width && py < cam.height;
  int region = inside ? rmap[(int64_t)py * cam.width + px] : -1;
  if (region >= R_total) { atomicOr(&hdr->status, kStatDeviceCheck); region = -1; }
  const float fpx = (float)px, fpy = (float)py;

  // ---- distinct regions of the tile -> slots ----
  {
    const unsigned peers = __match_any_sync(kFull, region);
    const bool leader = region >= 0 && lane == __ffs(peers) - 1;
    const unsigned leaders = __ballot_sync(kFull, leader);
    if (leader) sm.warp_regions[warp][__popc(leaders & ((1u << lane) - 1u))] = region;
    if (lane == 0) sm.warp_nreg[warp] = __popc(leaders);
  }
  for (int k = tid; k < kThreads * kMaxSlots; k += kThreads) (&sm.part[0][0])[k] = 0.0f;
  if (tid < 4) sm.cnt[tid] = 0ull;
  __syncthreads();
  if (tid == 0) {
    int ns = 0;
    for (int w = 0; w < kThreads / 32; ++w)
      for (int k = 0; k < sm.warp_nreg[w]; ++k) {
        const int r = sm.warp_regions[w][k];
        bool found = false;
        for (int q = 0; q < ns; ++q) found |= sm.slot_region[q] == r;
        if (!found && ns < kMaxSlots) sm.slot_region[ns++] = r;
      }
    sm.nslots = ns;
  }
  __syncthreads();
  const int nslots = sm.nslots;
  for (int k = tid; k < nslots * s; k += kThreads) {
    const int q = k / s, a = k - q * s;
    const int64_t row = (int64_t)sm.slot_region[q] * s + a;
    int j = code_idx[row];
    if (j >= C) { atomicOr(&hdr->status, kStatDeviceCheck); j = -1; }
    sm.slot_idx[q][a] = j;
    sm.slot_val[q][a] = code_val[row];
  }
  int my_slot = -1;
  for (int q = 0; q < nslots; ++q)
    if (sm.slot_region[q] == region) my_slot = q;
  const bool warp_uniform = __all_sync(kFull, region == __shfl_sync(kFull, region, 0));
  __syncthreads();

  float T = 1.0f;
  bool done = !inside;
  unsigned long long n_eval = 0, n_contrib = 0, n_flush = 0, n_atom = 0;

  unsigned long long last = 0ull;
  bool first = true;
  int remaining = n;
  bool all_done = false;
  while (!all_done && remaining > 0) {
    // ---- window of the kWin smallest remaining keys ----
    unsigned long long hi = ~0ull;
    if (remaining > kWin) hi = select_rank(sm, tkeys, n, last, first, kWin - 1);
    if (tid == 0) sm.cursor = 0u;
    __syncthreads();
    for (int i = tid; i < n; i += kThreads) {
      const unsigned long long k = tkeys[i];
      if ((first || k > last) && k <= hi) {
        const unsigned pos = atomicAdd(&sm.cursor, 1u);
        if (pos < (unsigned)kWin) sm.win[pos] = k;
      }
    }
    __syncthreads();
    const int m = (int)min(sm.cursor, (unsigned)kWin);
    if (m == 0 || sm.cursor > (unsigned)kWin) {
      // cannot happen for unique keys; stop this tile and report it
      if (tid == 0) atomicOr(&hdr->status, kStatDeviceCheck);
      break;
    }
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = m + tid; i < P; i += kThreads) sm.win[i] = ~0ull;
    __syncthreads();
    bitonic_sort(sm.win, P);
    const unsigned long long wlast = sm.win[m - 1];

    // ---- composite the window in batches ----
    for (int b0 = 0; b0 < m && !all_done; b0 += kThreads) {
      const int cnt = min(kThreads, m - b0);
      if (tid < cnt) {
        const int g = (int)(sm.win[b0 + tid] & 0xffffffffull);
        const ProjRec pr = proj[g];
        sm.rec_a[tid] = pr.a;
        sm.rec_b[tid] = pr.b;
        sm.gid[tid] = g;
      }
      __syncthreads();
      for (int j = 0; j < cnt; ++j) {
        float e = 0.0f;
        if (!done) {
          const float4 a = sm.rec_a[j];
          const float4 b = sm.rec_b[j];
          const float dx = a.x - fpx, dy = a.y - fpy;
          // power = dx*(qa*dx + qb*dy) + (qc*dy)*dy, products rounded, two fused sums
          const float power = fmaf(dx, fmaf(a.z, dx, __fmul_rn(a.w, dy)), __fmul_rn(__fmul_rn(b.x, dy), dy));
          ++n_eval;
          if (power <= 0.0f && power >= b.z) {
            const float alpha = fminf(0.99f, b.y * __expf(power));
            const float test = T * (1.0f - alpha);
            if (test < 1e-4f) {
              done = true;
            } else {
              e = alpha * T;
              T = test;
              ++n_contrib;
            }
          }
        }
        if (__any_sync(kFull, e > 0.0f)) {
          if (warp_uniform && my_slot >= 0) {
            const float ssum = warp_sum(e);
            if (lane == 0) atomicAdd(&sm.part[j][my_slot], ssum);
          } else if (e > 0.0f) {
            if (my_slot >= 0) {
              atomicAdd(&sm.part[j][my_slot], e);
            } else if (region >= 0) {
              // more regions in this tile than slots: scatter this pixel directly
              const int g = sm.gid[j];
              for (int a = 0; a < s; ++a) {
                const int64_t row = (int64_t)region * s + a;
                const int jj = code_idx[row];
                if (jj >= 0 && jj < C) {
                  atomicAdd(&accum[(int64_t)g * C + jj], code_val[row] * e);
                  ++n_atom;
                }
              }
              ++n_flush;
            }
          }
        }
      }
      __syncthreads();
      // ---- flush the (Gaussian, region) tile partials of this batch ----
      if (tid < cnt) {
        const int64_t g = sm.gid[tid];
        for (int q = 0; q < nslots; ++q) {
          const float v = sm.part[tid][q];
          if (v > 0.0f) {
            for (int a = 0; a < s; ++a) {
              const int jj = sm.slot_idx[q][a];
              if (jj >= 0) { atomicAdd(&accum[g * C + jj], sm.slot_val[q][a] * v); ++n_atom; }
            }
            ++n_flush;
            sm.part[tid][q] = 0.0f;
          }
        }
      }
      all_done = __syncthreads_and(done) != 0;
    }
    remaining -= m;
    last = wlast;
    first = false;
    __syncthreads();
  }

  // ---- counters ----
  for (int off = 16; off > 0; off >>= 1) {
    n_eval += __shfl_xor_sync(kFull, n_eval, off);
    n_contrib += __shfl_xor_sync(kFull, n_contrib, off);
    n_flush += __shfl_xor_sync(kFull, n_flush, off);
    n_atom += __shfl_xor_sync(kFull, n_atom, off);
  }
  if (lane == 0) {
    atomicAdd(&sm.cnt[0], n_eval);
    atomicAdd(&sm.cnt[1], n_contrib);
    atomicAdd(&sm.cnt[2], n_flush);
    atomicAdd(&sm.cnt[3], n_atom);
  }
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&hdr->evaluated, sm.cnt[0]);
    atomicAdd(&hdr->contributions, sm.cnt[1]);
    atomicAdd(&hdr->flushes, sm.cnt[2]);
    atomicAdd(&hdr->atomics, sm.cnt[3]);
  }
}

}  // namespace

cudaError_t launch_uplift_tiles(const CamArgs& cam, const UpliftWs& ws, const int32_t* rmap,
                                int32_t R_total, const int32_t* code_idx, const float* code_val,
                                int s, int C, float* accum, cudaStream_t st) {
  const int ntiles = cam.gx * cam.gy;
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = sizeof(TileSmem);
  cudaError_t err = cudaFuncSetAttribute(uplift_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  uplift_tile_kernel<<<ntiles, kThreads, smem, st>>>(cam, ws.proj, ws.keys, ws.tile_start, rmap,
                                                     R_total, code_idx, code_val, s, C, accum, ws.hdr);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace scoup
