// uplift_tile.cu -- per-tile front-to-back compositing and sparse scatter
// (paper Sec. 3 Eq. 2; Sec. 4.2 Eq. 5; Algorithm 1).
//
// One CTA per 16x16 tile, one pixel per thread; each warp covers a kBW x
// (32 / kBW) pixel block (8x4 by default; 16x2 and 4x8 are the other shapes
// the autotuner may pick).  The shape changes only which pixels share a warp
// (and so the order of the FP32 sums): membership is always decided on the
// 16x16 tile.
//
// Ordering.  The tile's key list (depth bits << 32 | Gaussian id, unordered)
// is read twice: a histogram pass over kNB depth buckets (a monotone map of
// the depth bits onto the view's depth range), then, per window of whole
// buckets holding at most kWin keys, a gather pass that places every key at
// its bucket's slot (a counting sort by bucket).  Inside a bucket the keys are
// ordered by rank (count of smaller keys in the same bucket, permuted in
// place), which gives the exact (depth, id) order.  A bucket holding more than kWin keys is split by a
// block-wide radix select.  Windows are composited front to back and the tile
// stops once every pixel has reached the transmittance cutoff, so the far part
// of a long list is never ordered.
//
// Scatter.  Codes are constant per region (Sec. 4.1), so the weights of all
// pixels of one region inside the tile are summed per Gaussian before the
// code is applied (distributivity): acc[g][j] += c_j * sum_p e_g(p).  A warp
// whose 32 pixels share one region reduces 8 Gaussians at a time with a
// transpose reduction (9 shuffles for 8 sums); other warps add per lane.  The
// per-(region, Gaussian) tile partials live in shared memory and are flushed
// as s global atomics once per window.
//
// Compensated form (kComp).  Every FP32 addition into the tile partials and
// into the global accumulator goes through an atomic that returns the old
// value; the rounding error of that addition is recovered exactly with
// Knuth's TwoSum (the atomic rounds to nearest, like the thread's own add) and
// added to a companion array (shared memory for the partials, accum + n*C in
// global memory), together with the exact error of the product c * e
// (fma(c, e, -c*e)).  The value of an entry is then sum + compensation.
//
// Semantic levels (kL = 3).  With several levels a pixel's region is the
// tuple of its regions in every level (packed 21 bits per level, 0 = none),
// a slot's code is the concatenation of the levels' codes with level l's
// atoms offset by l C, and the accumulator rows hold L C columns: one
// compositing pass scatters every level (the composite does not depend on
// the level).
//
// Load balance.  After the block-wide ordering of a window, each warp walks
// it independently (records staged per warp, no block barrier) and leaves as
// soon as its 32 pixels are saturated; the block meets again only at the end
// of the window.
//
// Depth slabs.  With several slabs per view the kernel runs once per slab;
// each pixel's transmittance (or its stop) is carried from one slab to the
// next in pix_state, and a tile whose pixels have all stopped is marked done:
// it returns at once in later slabs, and binning lists nothing for it.
#include <math.h>
#include <string.h>

#include "scoup_internal.cuh"

namespace scoup {
namespace {

constexpr int kThreads = 256;
static_assert(kThreads / 32 == 8, "one 8-bit block mask per record: eight warps per tile");
// Window of 256 keys over 1024 depth buckets: most pixels saturate within the
// first ~200 entries of a tile (1M-Gaussian views), so ordering more per
// window is mostly wasted; measured against 512/1024-key windows and 512/2048
// buckets, and against 5-6 CTAs per SM bought with register spills.
constexpr int kWin = 256;
constexpr int kLogNB = 10;
constexpr int kNB = 1 << kLogNB;
constexpr int kMaxSlots = 4;
constexpr int kMaxS = 64;  // codes of up to kMaxS entries are staged in shared memory; longer
                           // ones (dense features, Eq. 3) are read from the code table in the flush
constexpr int kGroup = 8;
// Each warp compacts the window entries whose box mask has its bit (up to
// kCompact at a time) and composites that list in full groups of kGroup.
constexpr int kCompact = kWin;
constexpr unsigned kFull = 0xffffffffu;
constexpr float kLog2e = 1.4426950408889634f;

// Region of a pixel: the region id (one level) or the packed level tuple.
template <int kL> struct RegionKey { using T = int; };
template <> struct RegionKey<3> { using T = unsigned long long; };
__device__ __forceinline__ bool region_set(int r) { return r >= 0; }
__device__ __forceinline__ bool region_set(unsigned long long r) { return r != 0ull; }
__device__ __forceinline__ int level_region(unsigned long long key, int l) {
  return (int)((key >> (21 * l)) & 0x1fffffull) - 1;
}

template <bool kComp, int kL>
struct TileSmem {
  uint32_t bstart[kNB + 1];
  uint32_t bcur[kNB];
  unsigned long long win[kWin];
  float4 rec_a[kWin + 1];  // the window's projected records, loaded once per window; entry kWin is
  float4 rec_b[kWin + 1];  // a record no pixel accepts (pads the warps' lists to whole groups)
  int wlist[kThreads / 32][kCompact + kGroup];  // per warp: window entries that may reach its pixels
  uint8_t rec_mask[kWin];  // per window entry: the warps whose pixel block it may reach
  float part[kMaxSlots][kWin];
  float part_c[kComp ? kMaxSlots : 1][kComp ? kWin : 1];
  uint8_t nzb[kMaxSlots][kWin];  // window entries whose partial became non-zero (plain byte stores)
  int flist[kThreads / 32][32];  // per warp: the marked entries of one mask word, in order
  typename RegionKey<kL>::T slot_region[kMaxSlots];
  int slot_idx[kMaxSlots][kMaxS];
  float slot_val[kMaxSlots][kMaxS];
  typename RegionKey<kL>::T warp_regions[kThreads / 32][32];
  int warp_nreg[kThreads / 32];
  uint32_t hist[256];
  unsigned long long red_min, red_max;
  unsigned int cursor;
  int nslots;
  int sel_digit;
  int sel_rank;
  int win_b1;
  unsigned long long cnt[4];
};

struct Buckets {
  uint32_t dmin;
  int shift;
  // monotone in the key and always inside [0, kNB)
  __device__ __forceinline__ int operator()(unsigned long long key) const {
    const uint32_t d = (uint32_t)(key >> 32);
    return (int)min((d > dmin ? d - dmin : 0u) >> shift, (uint32_t)(kNB - 1));
  }
};

// Block-wide: the rank-th smallest (0-based) key among those in bucket b
// with (first || key > last).  Keys are unique; requires rank < their count.
template <class Smem>
__device__ unsigned long long select_in_bucket(Smem& sm, const unsigned long long* __restrict__ keys,
                                               int n, const Buckets& bk, int b, unsigned long long last,
                                               bool first, int rank) {
  const int tid = threadIdx.x;
  if (tid == 0) { sm.red_min = ~0ull; sm.red_max = 0ull; }
  __syncthreads();
  unsigned long long lmin = ~0ull, lmax = 0ull;
  for (int i = tid; i < n; i += kThreads) {
    const unsigned long long k = keys[i];
    if (bk(k) == b && (first || k > last)) { lmin = min(lmin, k); lmax = max(lmax, k); }
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
      if (bk(k) == b && (first || k > last)) {
        const unsigned long long x = k - base;
        if ((x & pmask) == prefix) atomicAdd(&sm.hist[(x >> shift) & 255u], 1u);
      }
    }
    __syncthreads();
    if (tid < 32) {
      uint32_t c[8], sum = 0;
      for (int d = 0; d < 8; ++d) { c[d] = sm.hist[tid * 8 + d]; sum += c[d]; }
      uint32_t incl = sum;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, off);
        if (tid >= off) incl += y;
      }
      const uint32_t excl = incl - sum;
      if ((uint32_t)rank >= excl && (uint32_t)rank < incl) {
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

// Reduce 8 per-lane values across the warp: every lane ends up holding the
// sum over all 32 lanes of v[lane >> 2].
__device__ __forceinline__ float transpose_reduce8(const float (&v)[kGroup], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b4 ? v[4 + i] : v[i];
    const float send = b4 ? v[i] : v[4 + i];
    a[i] = keep + __shfl_xor_sync(kFull, send, 16);
  }
  float c[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b3 ? a[2 + i] : a[i];
    const float send = b3 ? a[i] : a[2 + i];
    c[i] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  float d = (b2 ? c[1] : c[0]) + __shfl_xor_sync(kFull, b2 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(kFull, d, 2);
  d += __shfl_xor_sync(kFull, d, 1);
  return d;
}

// 2^x by the SFU's approximate base-2 exponential (relative error about
// 2^-22; results below the smallest normal flush to zero, far below any
// accepted alpha).
__device__ __forceinline__ float exp2f_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Error of s = fl(a + b) (Knuth's TwoSum): a + b = s + err exactly.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  return __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// part[i] += v (v > 0, shared memory), compensated when kComp; every
// addition marks the entry for the flush with a plain byte store (all
// writers store the same 1, so no atomic is needed).  The plain form never
// reads the atomic's result, so the warp does not wait for it.
template <bool kComp>
__device__ __forceinline__ void part_add(float* part, float* part_c, uint8_t* nzb, int i, float v) {
  nzb[i] = 1;
  if constexpr (kComp) {
    const float old = atomicAdd(&part[i], v);
    const float err = two_sum_err(old, v, __fadd_rn(old, v));
    if (err != 0.0f) atomicAdd(&part_c[i], err);
  } else {
    atomicAdd(&part[i], v);
  }
}

// accum[x] += c * (v + vc) (global memory), compensated when kComp (vc is the
// compensation of v; 0 in the plain form).
template <bool kComp>
__device__ __forceinline__ void acc_add(float* accum, float* comp, int64_t x, float c, float v, float vc) {
  if constexpr (!kComp) {
    atomicAdd(&accum[x], c * v);
  } else {
    const float p = __fmul_rn(c, v);
    const float perr = __fmaf_rn(c, v, -p);  // c * v - p exactly
    const float old = atomicAdd(&accum[x], p);
    const float err = __fadd_rn(__fadd_rn(two_sum_err(old, p, __fadd_rn(old, p)), perr), __fmul_rn(c, vc));
    if (err != 0.0f) atomicAdd(&comp[x], err);
  }
}

// The whole pass over one tile of one view: ordering, compositing, flush and
// counters.  Called by the per-view kernel (one CTA per tile) and by the
// batched drain kernel (a CTA takes tiles of several views in turn); every
// early return is taken by the whole CTA.
template <bool kComp, int kBW, int kL>
__device__ __forceinline__ void tile_pass(
    TileSmem<kComp, kL>& sm, const int tile, const CamArgs& cam, const ProjRec* __restrict__ proj,
    const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ tile_start, int slot,
    const LevelCodes& lc, int C, int Crow, float* __restrict__ accum, float* __restrict__ comp,
    WsHeader* __restrict__ hdr, float* __restrict__ pix_state, uint8_t* __restrict__ tile_done, int slab,
    int nslabs) {
  const bool first_slab = slab == 0, last_slab = slab == nslabs - 1;
  using RK = typename RegionKey<kL>::T;
  // code entries per slot (the concatenated level codes with several levels)
  const int s = kL == 1 ? lc.s[0] : lc.s_tot;
  const int32_t* __restrict__ code_idx = lc.ci[0];
  const float* __restrict__ code_val = lc.cv[0];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (pix_state && !first_slab && tile_done[tile]) return;  // every pixel stopped in an earlier slab
  const uint32_t begin = tile_start[tile];
  const int n = (int)(tile_start[tile + 1] - begin);
  if (n == 0) return;  // nothing of this slab here: the pixels' state stays as it is
  if (hdr->status & kStatCapacity) return;
  const unsigned long long* tkeys = keys + begin;

  Buckets bk;
  {
    // the buckets span the view's visible depths, cut to this slab's range
    uint32_t dmin = hdr->drange[slot][0], dmax = hdr->drange[slot][1];
    if (nslabs > 1) {
      dmin = max(dmin, hdr->slab_lo[slot][slab]);
      if (!last_slab && hdr->slab_lo[slot][slab + 1] > 0u) dmax = min(dmax, hdr->slab_lo[slot][slab + 1] - 1u);
    }
    const uint32_t span = dmax >= dmin ? dmax - dmin : 0u;
    const int nb = span ? 32 - __clz((int)span) : 0;
    bk.dmin = dmin;
    bk.shift = nb > kLogNB ? nb - kLogNB : 0;
  }

  const int tx = tile % cam.gx, ty = tile / cam.gx;
  constexpr int kBH = 32 / kBW, kWarpsX = kTile / kBW;
  const int bxi = tx * kTile + (warp % kWarpsX) * kBW, byi = ty * kTile + (warp / kWarpsX) * kBH;
  const int px = bxi + lane % kBW;
  const int py = byi + lane / kBW;
  const bool inside = px < cam.width && py < cam.height;
  RK region;
  if constexpr (kL == 1) {
    int r = inside ? lc.rmap[0][(int64_t)py * cam.width + px] : -1;
    if (r >= lc.R[0]) { atomicOr(&hdr->status, kStatDeviceCheck); r = -1; }
    region = r;
  } else {
    unsigned long long key = 0ull;
    for (int l = 0; l < lc.L; ++l) {
      int r = inside ? lc.rmap[l][(int64_t)py * cam.width + px] : -1;
      if (r >= lc.R[l]) { atomicOr(&hdr->status, kStatDeviceCheck); r = -1; }
      if (r >= 0) key |= (unsigned long long)(r + 1) << (21 * l);
    }
    region = key;
  }
  const float fpx = (float)px, fpy = (float)py;

  // ---- distinct regions of the tile -> slots; bucket histogram ----
  {
    const unsigned peers = __match_any_sync(kFull, region);
    const bool leader = region_set(region) && lane == __ffs(peers) - 1;
    const unsigned leaders = __ballot_sync(kFull, leader);
    if (leader) sm.warp_regions[warp][__popc(leaders & ((1u << lane) - 1u))] = region;
    if (lane == 0) sm.warp_nreg[warp] = __popc(leaders);
  }
  for (int k = tid; k < kMaxSlots * kWin; k += kThreads) (&sm.part[0][0])[k] = 0.0f;
  if constexpr (kComp)
    for (int k = tid; k < kMaxSlots * kWin; k += kThreads) (&sm.part_c[0][0])[k] = 0.0f;
  for (int k = tid; k < kMaxSlots * kWin / 4; k += kThreads) reinterpret_cast<uint32_t*>(&sm.nzb[0][0])[k] = 0u;
  if (tid == 0) {
    // power = 0 for any pixel, never >= tau = +inf: no pixel accepts it
    sm.rec_a[kWin] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    sm.rec_b[kWin] = make_float4(0.0f, 0.0f, INFINITY, 0.0f);
  }
  for (int b = tid; b < kNB; b += kThreads) sm.bcur[b] = 0u;
  if (tid < 4) sm.cnt[tid] = 0ull;
  __syncthreads();
  for (int i = tid; i < n; i += kThreads) atomicAdd(&sm.bcur[bk(tkeys[i])], 1u);
  if (tid == 0) {
    int ns = 0;
    for (int w = 0; w < kThreads / 32; ++w)
      for (int k = 0; k < sm.warp_nreg[w]; ++k) {
        const RK r = sm.warp_regions[w][k];
        bool found = false;
        for (int q = 0; q < ns; ++q) found |= sm.slot_region[q] == r;
        if (!found && ns < kMaxSlots) sm.slot_region[ns++] = r;
      }
    sm.nslots = ns;
  }
  __syncthreads();
  // exclusive scan of the bucket counts (kNB / kThreads per thread, then across warps)
  {
    constexpr int kPer = kNB / kThreads;
    uint32_t c[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) { c[q] = sm.bcur[tid * kPer + q]; sum += c[q]; }
    uint32_t incl = sum;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, off);
      if (lane >= off) incl += y;
    }
    if (lane == 31) sm.hist[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += sm.hist[w];
    uint32_t run = wbase + incl - sum;
#pragma unroll
    for (int q = 0; q < kPer; ++q) { sm.bstart[tid * kPer + q] = run; run += c[q]; }
    if (tid == kThreads - 1) sm.bstart[kNB] = run;
  }
  const int nslots = sm.nslots;
  for (int k = tid; k < (s <= kMaxS ? nslots * s : 0); k += kThreads) {
    const int q = k / s, a = k - q * s;
    if constexpr (kL == 1) {
      const int64_t row = (int64_t)sm.slot_region[q] * s + a;
      int j = code_idx[row];
      if (j >= C) { atomicOr(&hdr->status, kStatDeviceCheck); j = -1; }
      sm.slot_idx[q][a] = j;
      sm.slot_val[q][a] = code_val[row];
    } else {
      int l = 0, e = a;  // level of entry a and its index in that level's code
      while (l < lc.L - 1 && e >= lc.s[l]) { e -= lc.s[l]; ++l; }
      const int r = level_region(sm.slot_region[q], l);
      int j = -1;
      float v = 0.0f;
      if (r >= 0) {
        const int64_t row = (int64_t)r * lc.s[l] + e;
        j = lc.ci[l][row];
        v = lc.cv[l][row];
        if (j >= C) { atomicOr(&hdr->status, kStatDeviceCheck); j = -1; }
        if (j >= 0) j += l * C;
      }
      sm.slot_idx[q][a] = j;
      sm.slot_val[q][a] = v;
    }
  }
  int my_slot = -1;
  for (int q = 0; q < nslots; ++q)
    if (sm.slot_region[q] == region) my_slot = q;
  const bool uniform = __all_sync(kFull, region == __shfl_sync(kFull, region, 0));
  const int wslot = uniform ? my_slot : -1;
  // slots present among the warp's pixels, and whether some pixel's region got no slot
  unsigned wslots = 0u;
  for (int q = 0; q < nslots; ++q)
    if (__any_sync(kFull, my_slot == q)) wslots |= 1u << q;
  const bool any_unslotted = __any_sync(kFull, my_slot < 0 && region_set(region));
  __syncthreads();

  float T = 1.0f;
  bool done = !inside;
  if (pix_state && !first_slab) {
    const float sv = pix_state[(int64_t)tile * kTilePixels + tid];
    if (sv < 0.0f) done = true;
    else if (sv > 0.0f) T = sv;
  }
  unsigned n_eval = 0, n_contrib = 0, n_flush = 0, n_atom = 0;  // per thread and tile: fits 32 bits

  int b0 = 0;
  bool all_done = false;
  // a bucket holding more than kWin keys is consumed in sub-windows
  bool in_split = false, split_first = true;
  unsigned long long split_last = 0ull;
  int consumed = 0;
  while (!all_done && b0 < kNB) {
    const uint32_t base = sm.bstart[b0];
    const int total_b0 = (int)(sm.bstart[b0 + 1] - base);
    if (!in_split && total_b0 == 0) {
      // skip empty buckets quickly: find the next non-empty one
      if (tid == 0) {
        int lo = b0 + 1, hi = kNB;  // smallest b with bstart[b + 1] > base, i.e. first b with keys
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sm.bstart[mid + 1] > base) hi = mid; else lo = mid + 1;
        }
        sm.win_b1 = lo;
      }
      __syncthreads();
      b0 = sm.win_b1;
      __syncthreads();
      continue;
    }
    if (!in_split) {
      if (tid == 0) {
        // largest b1 in [b0 + 1, kNB] with bstart[b1] - base <= kWin (b0 itself if it is oversize)
        int lo = b0 + 1, hi = kNB;
        if (sm.bstart[lo] - base > (uint32_t)kWin) {
          sm.win_b1 = b0;
        } else {
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.bstart[mid] - base <= (uint32_t)kWin) lo = mid; else hi = mid - 1;
          }
          sm.win_b1 = lo;
        }
      }
      __syncthreads();
    }
    const int b1 = sm.win_b1;
    int m;
    if (!in_split && b1 > b0) {
      // ---- gather whole buckets [b0, b1) at their slots, rank inside buckets ----
      m = (int)(sm.bstart[b1] - base);
      for (int b = b0 + tid; b < b1; b += kThreads) sm.bcur[b] = sm.bstart[b] - base;
      __syncthreads();
      for (int i = tid; i < n; i += kThreads) {
        const unsigned long long k = tkeys[i];
        const int b = bk(k);
        if (b >= b0 && b < b1) {
          const uint32_t pos = atomicAdd(&sm.bcur[b], 1u);
          if (pos < (uint32_t)kWin) sm.win[pos] = k;
        }
      }
      __syncthreads();
      // rank inside the bucket, then permute in place (keys held in registers)
      unsigned long long kk[kWin / kThreads];
      int dst[kWin / kThreads];
#pragma unroll
      for (int u = 0; u < kWin / kThreads; ++u) {
        const int p = tid + u * kThreads;
        dst[u] = -1;
        if (p < m) {
          const unsigned long long k = sm.win[p];
          const int b = bk(k);
          const int lo = (int)(sm.bstart[b] - base), hi = (int)(sm.bstart[b + 1] - base);
          int r = 0;
          for (int q = lo; q < hi; ++q) r += sm.win[q] < k;
          kk[u] = k;
          dst[u] = lo + r;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kWin / kThreads; ++u)
        if (dst[u] >= 0) sm.win[dst[u]] = kk[u];
    } else {
      // ---- oversize bucket b0: the kWin smallest of its remaining keys ----
      if (!in_split) { in_split = true; split_first = true; consumed = 0; }
      if (tid == 0) atomicAdd(&hdr->split_windows, 1ull);
      const int left = total_b0 - consumed;
      unsigned long long hi_key = ~0ull;
      if (left > kWin) hi_key = select_in_bucket(sm, tkeys, n, bk, b0, split_last, split_first, kWin - 1);
      if (tid == 0) sm.cursor = 0u;
      __syncthreads();
      for (int i = tid; i < n; i += kThreads) {
        const unsigned long long k = tkeys[i];
        if (bk(k) == b0 && (split_first || k > split_last) && k <= hi_key) {
          const unsigned pos = atomicAdd(&sm.cursor, 1u);
          if (pos < (unsigned)kWin) sm.win[pos] = k;
        }
      }
      __syncthreads();
      m = (int)min(sm.cursor, (unsigned)kWin);
      unsigned long long kk[kWin / kThreads];
      int dst[kWin / kThreads];
#pragma unroll
      for (int u = 0; u < kWin / kThreads; ++u) {
        const int p = tid + u * kThreads;
        dst[u] = -1;
        if (p < m) {
          const unsigned long long k = sm.win[p];
          int r = 0;
          for (int q = 0; q < m; ++q) r += sm.win[q] < k;
          kk[u] = k;
          dst[u] = r;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kWin / kThreads; ++u)
        if (dst[u] >= 0) sm.win[dst[u]] = kk[u];
    }
    __syncthreads();
    if (m <= 0) {
      if (tid == 0) atomicOr(&hdr->status, kStatDeviceCheck);
      break;
    }

    // ---- composite the window: every warp walks it on its own ----
    // The CTA loads the window's records into shared memory once (one per
    // thread, all loads in flight together), and the same thread marks which
    // of the tile's eight warp blocks the record may reach (box_grid_mask).
    // Each warp composites only the Gaussians whose mark has its bit, in
    // window order.
    for (int j = tid; j < m; j += kThreads) {
      const ProjRec pr = proj[(int)(sm.win[j] & 0xffffffffull)];
      sm.rec_a[j] = pr.a;
      sm.rec_b[j] = pr.b;
      sm.rec_mask[j] = (uint8_t)box_grid_mask<kWarpsX, kTile / kBH>(pr, (float)(tx * kTile), (float)(ty * kTile),
                                                                   (float)kBW, (float)kBH);
    }
    __syncthreads();
    bool warp_done = __all_sync(kFull, done);
    const float4* st_a = sm.rec_a;
    const float4* st_b = sm.rec_b;
    int* wl = sm.wlist[warp];
    for (int c0 = 0; c0 < m && !warp_done; c0 += kCompact) {
      // box test of the next kCompact records; the warp's list keeps, in
      // window order, the entries that may reach one of its pixels, padded
      // with the dummy entry kWin to whole groups
      const int c1 = min(m, c0 + kCompact);
      int cnt = 0;
      for (int j0 = c0; j0 < c1; j0 += 32) {
        const int j = j0 + lane;
        const bool rel = j < c1 && ((sm.rec_mask[j] >> warp) & 1u);
        const unsigned rmask = __ballot_sync(kFull, rel);
        if (rel) wl[cnt + __popc(rmask & ((1u << lane) - 1u))] = j;
        cnt += __popc(rmask);
      }
      if (lane < kGroup) wl[cnt + lane] = kWin;
      __syncwarp();
      for (int g0 = 0; g0 < cnt && !warp_done; g0 += kGroup) {
        const int* idx = wl + g0;  // this group's window entries (read per slot: fewer live registers)
        // slots of this group this pixel examines: all real ones while it is
        // open, up to and including the one at which it stops
        int ev = done ? 0 : min(kGroup, cnt - g0);
        float e[kGroup];
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
          const float4 a = st_a[idx[u]];
          const float4 b = st_b[idx[u]];
          const float dx = a.x - fpx, dy = a.y - fpy;
          // power = dx*(qa*dx + qb*dy) + (qc*dy)*dy: products rounded, two fused sums
          const float power = fmaf(dx, fmaf(a.z, dx, __fmul_rn(a.w, dy)), __fmul_rn(__fmul_rn(b.x, dy), dy));
          const bool accept = !done && power <= 0.0f && power >= b.z;
          // alpha = min(0.99, o exp(power)) = min(0.99, 2^(power log2(e) + log2(o))), b.w = log2(o)
          const float alpha = fminf(0.99f, exp2f_approx(fmaf(power, kLog2e, b.w)));
          const float test = fmaf(-T, alpha, T);  // T (1 - alpha)
          const bool stop = accept && test < 1e-4f;
          const bool take = accept && !stop;
          e[u] = take ? alpha * T : 0.0f;
          T = take ? test : T;
          ev = stop ? u + 1 : ev;
          done = done || stop;
          n_contrib += take ? 1u : 0u;
        }
        n_eval += (unsigned)ev;
        // Gaussian of this lane's quarter of the reduction (its window entry)
        const int jq = wl[g0 + (lane >> 2)];
        if (wslot >= 0) {
          const float S = transpose_reduce8(e, lane);
          if ((lane & 3) == 0 && S > 0.0f)
            part_add<kComp>(sm.part[wslot], sm.part_c[kComp ? wslot : 0], sm.nzb[wslot], jq, S);
        } else {
          // pixels of several regions: one masked transpose reduction per slot present
          for (unsigned qm = wslots; qm != 0u; qm &= qm - 1u) {
            const int q = __ffs(qm) - 1;
            float v[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u) v[u] = my_slot == q ? e[u] : 0.0f;
            const float S = transpose_reduce8(v, lane);
            if ((lane & 3) == 0 && S > 0.0f)
              part_add<kComp>(sm.part[q], sm.part_c[kComp ? q : 0], sm.nzb[q], jq, S);
          }
          if (any_unslotted && my_slot < 0 && region_set(region)) {
            // more regions in this tile than slots: scatter this pixel directly
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
              if (!(e[u] > 0.0f)) continue;
              const int64_t g = (int64_t)(sm.win[idx[u]] & 0xffffffffull);
              for (int l = 0; l < (kL == 1 ? 1 : lc.L); ++l) {
                int r;
                if constexpr (kL == 1) r = region; else r = level_region(region, l);
                if (r < 0) continue;
                for (int a = 0; a < lc.s[l]; ++a) {
                  const int64_t row = (int64_t)r * lc.s[l] + a;
                  const int jj = lc.ci[l][row];
                  if (jj >= C) atomicOr(&hdr->status, kStatDeviceCheck);
                  if (jj >= 0 && jj < C) {
                    acc_add<kComp>(accum, comp, g * Crow + l * C + jj, lc.cv[l][row], e[u], 0.0f);
                    ++n_atom;
                  }
                }
              }
              ++n_flush;
            }
          }
        }
        warp_done = __all_sync(kFull, done);
      }
      __syncwarp();  // the list is rewritten by the next batch
    }
    __syncthreads();
    // ---- flush the (region, Gaussian) tile partials of this window ----
    // A warp takes one 32-entry word of the marks at a time (window entries
    // [32 w, 32 w + 32) of one slot), compacts the marked entries into its
    // list and issues the atomics of 32 / min(s, 32) of them per step, one
    // code entry per lane; the first lane of an entry's group reads (and
    // clears) the partial and passes it on with a shuffle.  (Numbering the
    // marked entries across all warps balances better but costs more per
    // entry: measured slower.)
    const int nwords = (m + 31) >> 5;
    const int nw = nslots * nwords;
    {
      const int lanes_per = s < 32 ? s : 32;
      const int per = 32 / lanes_per;
      const int sub = lane / lanes_per, a0 = lane - sub * lanes_per;
      int* fl = sm.flist[warp];
      for (int wi = warp; wi < nw; wi += kThreads / 32) {
        const int q = wi / nwords, j = (wi - q * nwords) * 32 + lane;
        const bool f = sm.nzb[q][j] != 0;
        const unsigned bits = __ballot_sync(kFull, f);
        if (f) {
          fl[__popc(bits & ((1u << lane) - 1u))] = j;
          sm.nzb[q][j] = 0;
        }
        __syncwarp();
        const int cnt = __popc(bits);
        for (int k0 = 0; k0 < cnt; k0 += per) {
          const int k = k0 + sub;
          const bool act = sub < per && k < cnt;
          const int p = act ? fl[k] : 0;
          float v = 0.0f, vc = 0.0f;
          if (act && a0 == 0) {
            v = sm.part[q][p];
            sm.part[q][p] = 0.0f;
            if constexpr (kComp) {
              vc = sm.part_c[q][p];
              sm.part_c[q][p] = 0.0f;
            }
            ++n_flush;
          }
          v = __shfl_sync(kFull, v, sub * lanes_per);
          if constexpr (kComp) vc = __shfl_sync(kFull, vc, sub * lanes_per);
          if (act) {
            const int64_t g = (int64_t)(sm.win[p] & 0xffffffffull);
            for (int a = a0; a < s; a += lanes_per) {
              int jj;
              float cval;
              if (kL > 1 || s <= kMaxS) {
                jj = sm.slot_idx[q][a];
                cval = sm.slot_val[q][a];
              } else {
                const int64_t row = (int64_t)sm.slot_region[q] * s + a;
                jj = code_idx[row];
                cval = code_val[row];
                if (jj >= C) { atomicOr(&hdr->status, kStatDeviceCheck); jj = -1; }
              }
              if (jj >= 0) { acc_add<kComp>(accum, comp, g * Crow + jj, cval, v, vc); ++n_atom; }
            }
          }
        }
        __syncwarp();  // the list is rewritten for the next word
      }
    }
    all_done = __syncthreads_and(done) != 0;

    // ---- advance to the next window ----
    if (in_split) {
      consumed += m;
      split_last = sm.win[m - 1];
      split_first = false;
      if (consumed >= total_b0) { in_split = false; b0 += 1; }
    } else {
      b0 = b1;
    }
    __syncthreads();
  }

  // ---- state for the next slab ----
  if (pix_state && !last_slab) {
    pix_state[(int64_t)tile * kTilePixels + tid] = done ? -1.0f : T;
    if (__syncthreads_and(done) && tid == 0) tile_done[tile] = 1;
  }

  // ---- counters ----
  for (int off = 16; off > 0; off >>= 1) {
    n_eval += __shfl_xor_sync(kFull, n_eval, off);
    n_contrib += __shfl_xor_sync(kFull, n_contrib, off);
    n_flush += __shfl_xor_sync(kFull, n_flush, off);
    n_atom += __shfl_xor_sync(kFull, n_atom, off);
  }
  if (lane == 0) {
    atomicAdd(&sm.cnt[0], (unsigned long long)n_eval);
    atomicAdd(&sm.cnt[1], (unsigned long long)n_contrib);
    atomicAdd(&sm.cnt[2], (unsigned long long)n_flush);
    atomicAdd(&sm.cnt[3], (unsigned long long)n_atom);
  }
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&hdr->evaluated, sm.cnt[0]);
    atomicAdd(&hdr->contributions, sm.cnt[1]);
    atomicAdd(&hdr->flushes, sm.cnt[2]);
    atomicAdd(&hdr->atomics, sm.cnt[3]);
  }
}

template <bool kComp, int kBW, int kL>
__global__ void __launch_bounds__(kThreads, kComp ? 3 : 4) uplift_tile_kernel(
    const __grid_constant__ CamArgs cam, const ProjRec* __restrict__ proj,
    const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ tile_start, int slot,
    const __grid_constant__ LevelCodes lc, int C, int Crow, float* __restrict__ accum, float* __restrict__ comp,
    WsHeader* __restrict__ hdr, float* __restrict__ pix_state, uint8_t* __restrict__ tile_done, int slab,
    int nslabs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_pass<kComp, kBW, kL>(*reinterpret_cast<TileSmem<kComp, kL>*>(smem_raw), blockIdx.x, cam, proj, keys,
                            tile_start, slot, lc, C, Crow, accum, comp, hdr, pix_state, tile_done, slab, nslabs);
}

// Batched chunk: a persistent CTA takes (view, tile) items from the chunk's
// counter until none is left and runs the same per-tile pass on each.  The
// chunk's views travel in the kernel's parameter space (like the per-view
// kernel's arguments, read through the constant cache), which keeps them out
// of the pass's registers.  No CTA waits on another.
struct DrainArgs {
  uint32_t tile0[kMaxDrainJobs];  // first item of each view (ascending, tile0[0] = 0)
  int njobs;
  uint32_t total;
  TileJob jobs[kMaxDrainJobs];
};
static_assert(sizeof(DrainArgs) <= 32000, "kernel parameter space");

template <bool kComp, int kBW>
__global__ void __launch_bounds__(kThreads, kComp ? 3 : 4) uplift_drain_kernel(const __grid_constant__ DrainArgs a,
                                                                             unsigned* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<kComp, 1>& sm = *reinterpret_cast<TileSmem<kComp, 1>*>(smem_raw);
  __shared__ uint32_t s_item;
  __shared__ int s_job;
  for (;;) {
    __syncthreads();  // the previous pass is done with the tile's shared memory
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(counter, 1u);
      int lo = 0;
      if (t < a.total) {
        int hi = a.njobs - 1;  // last view whose first item is at or before t
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.tile0[mid] <= t) lo = mid; else hi = mid - 1;
        }
      }
      s_item = t;
      s_job = lo;
    }
    __syncthreads();
    const uint32_t t = s_item;
    if (t >= a.total) return;
    const TileJob& job = a.jobs[s_job];
    tile_pass<kComp, kBW, 1>(sm, (int)(t - a.tile0[s_job]), job.cam, job.proj, job.keys, job.tile_start, job.slot,
                             job.lc, job.C, job.C, job.accum, job.comp, job.hdr, nullptr, nullptr, 0, 1);
  }
}

struct SlabLaunch {
  float* pix_state;  // null with a single slab
  uint8_t* tile_done;
  int slab, nslabs;
};

template <bool kComp, int kBW, int kL>
cudaError_t launch_tiles_t(const CamArgs& cam, const UpliftWs& ws, int slot, const LevelCodes& lc, int C, int Crow,
                           float* accum, float* comp, const SlabLaunch& sl, cudaStream_t st) {
  const int ntiles = cam.gx * cam.gy;
  const size_t smem = sizeof(TileSmem<kComp, kL>);
  cudaError_t err = cudaFuncSetAttribute(uplift_tile_kernel<kComp, kBW, kL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  uplift_tile_kernel<kComp, kBW, kL><<<ntiles, kThreads, smem, st>>>(
      cam, ws.proj, ws.keys, ws.tile_start, slot, lc, C, Crow, accum, comp, ws.hdr, sl.pix_state, sl.tile_done,
      sl.slab, sl.nslabs);
  g_launches += 1;
  return cudaGetLastError();
}

template <bool kComp>
cudaError_t launch_tiles_shape(int warp_w, const CamArgs& cam, const UpliftWs& ws, int slot, const LevelCodes& lc,
                               int C, int Crow, float* accum, float* comp, const SlabLaunch& sl, cudaStream_t st) {
  if (lc.L > 1) return launch_tiles_t<kComp, 8, 3>(cam, ws, slot, lc, C, Crow, accum, comp, sl, st);
  switch (warp_w) {
    case 16: return launch_tiles_t<kComp, 16, 1>(cam, ws, slot, lc, C, Crow, accum, comp, sl, st);
    case 4: return launch_tiles_t<kComp, 4, 1>(cam, ws, slot, lc, C, Crow, accum, comp, sl, st);
    default: return launch_tiles_t<kComp, 8, 1>(cam, ws, slot, lc, C, Crow, accum, comp, sl, st);
  }
}

template <bool kComp, int kBW>
cudaError_t launch_drain_t(const DrainArgs& args, unsigned* counter, cudaStream_t st) {
  const size_t smem = sizeof(TileSmem<kComp, 1>);
  auto kern = uplift_drain_kernel<kComp, kBW>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  // CTAs resident per SM by the launch bounds (the shared memory of four fits);
  // a CTA beyond them would only start later and drain what is left
  const long long resident = (long long)num_sms() * (kComp ? 3 : 4);
  const int grid = (int)(args.total < (uint32_t)resident ? args.total : (uint32_t)resident);
  kern<<<grid, kThreads, smem, st>>>(args, counter);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_uplift_drain(const TileJob* jobs, const uint32_t* tile0, int njobs, unsigned* counter,
                                bool compensated, int warp_w, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (njobs > kMaxDrainJobs) return cudaErrorInvalidValue;
  DrainArgs args;
  memset(&args, 0, sizeof(args));
  args.njobs = njobs;
  uint32_t total = 0;
  for (int j = 0; j < njobs; ++j) {
    if (tile0[j] != total) return cudaErrorInvalidValue;
    args.tile0[j] = tile0[j];
    args.jobs[j] = jobs[j];
    total += (uint32_t)jobs[j].tiles;
  }
  args.total = total;
  if (total == 0) return cudaSuccess;
  if (compensated) {
    switch (warp_w) {
      case 16: return launch_drain_t<true, 16>(args, counter, st);
      case 4: return launch_drain_t<true, 4>(args, counter, st);
      default: return launch_drain_t<true, 8>(args, counter, st);
    }
  }
  switch (warp_w) {
    case 16: return launch_drain_t<false, 16>(args, counter, st);
    case 4: return launch_drain_t<false, 4>(args, counter, st);
    default: return launch_drain_t<false, 8>(args, counter, st);
  }
}

cudaError_t launch_uplift_tiles(const CamArgs& cam, const UpliftWs& ws, int slot, const LevelCodes& lc, int C,
                                int Crow, float* accum, float* comp, int warp_w, cudaStream_t st, int slab,
                                int nslabs) {
  static_assert(sizeof(TileSmem<false, 1>) <= 55 * 1024, "4 CTAs per SM");
  static_assert(sizeof(TileSmem<false, 3>) <= 55 * 1024, "4 CTAs per SM");
  static_assert(sizeof(TileSmem<true, 3>) <= 74 * 1024, "3 CTAs per SM");
  if (cam.gx * cam.gy <= 0) return cudaSuccess;
  SlabLaunch sl;
  sl.pix_state = nslabs > 1 ? ws.pix_state : nullptr;
  sl.tile_done = ws.tile_done;
  sl.slab = nslabs > 1 ? slab : 0;
  sl.nslabs = nslabs > 1 ? nslabs : 1;
  if (comp) return launch_tiles_shape<true>(warp_w, cam, ws, slot, lc, C, Crow, accum, comp, sl, st);
  return launch_tiles_shape<false>(warp_w, cam, ws, slot, lc, C, Crow, accum, nullptr, sl, st);
}

}  // namespace scoup
