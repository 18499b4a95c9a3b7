// binning.cu -- tile binning of one view's projected Gaussians.
//
// Every visible Gaussian is listed in the 16x16 tiles of its rectangle (the
// 3DGS rule: membership is tile-granular).  The rectangles here are the 3DGS
// rectangles cut to the bounding box of each Gaussian's alpha >= 1/255
// ellipse (by the projection): a dropped tile holds no pixel that passes the
// alpha test, so the composite is unchanged.  The per-tile lists hold 64-bit
// keys (depth bits << 32 | original Gaussian index); they are left unordered
// here and ordered front to back (depth, then index) inside the tile kernel.
//
// The Gaussians arrive in spatial (Morton) order, so one CTA's chunk covers a
// compact block of tiles.  Each warp expands the (Gaussian, tile) items of its
// 32 Gaussians cooperatively, one item per lane per round.  Counting is
// privatised per CTA in shared memory over the chunk's tile bounding box; the
// counting pass reserves the CTA's run in each tile list right away (one
// global atomic per (CTA, tile)) and keeps the run's offset, so the filling
// pass expands the items only once and writes each CTA's keys of a tile into
// one contiguous run.  A warp whose rectangles overlap heavily walks their
// union tile by tile instead, so that the keys of one tile leave in one
// coalesced store.  Rectangles larger than kBigRect tiles go to separate
// global counters and are placed after the reserved runs.
//
// Depth slabs.  Called for slab s of a view, both passes take only the
// Gaussians whose depth lies in the slab, and for s > 0 only the tiles that
// still hold an open pixel: a Gaussian whose rectangle has no such tile is
// dropped before expansion, and items in done tiles are skipped.
#include "scoup_internal.cuh"

namespace scoup {
namespace {

// one Morton-ordered Gaussian per thread, 512 per CTA (measured fastest
// against 256..2048-Gaussian chunks and 64..512 threads on the 1M-Gaussian views)
constexpr int kBinThreads = 512;
constexpr int64_t kChunk = 512;
constexpr int kLocalMax = 4096;  // tiles of the per-CTA bounding box kept in shared memory
constexpr int kBigRect = 256;
// A warp's union path is taken when its items are at least this many times
// the tiles of its rectangles' union.  Measured on 1M-Gaussian 988x731 views
// over thresholds 1..32: 8 is best (fill 75 -> 67 us per view); lower ones let
// in warps whose per-tile loop costs more than the coalesced stores save, and
// from 12 up no warp qualifies.
constexpr int kUnionItemsPerTile = 8;
constexpr unsigned kFull = 0xffffffffu;

// Which Gaussians and tiles one binning call takes.
struct SlabSel {
  uint32_t lo, hi;       // depth bits [lo, hi) (hi unused when last)
  bool active, last;
  const uint8_t* done;   // tile done flags, or null (no tile is skipped)

  __device__ __forceinline__ bool skip_tile(int t) const { return done && done[t]; }
};

__device__ __forceinline__ SlabSel slab_sel(const WsHeader* __restrict__ hdr, int slot, int slab, int last,
                                            const uint8_t* done) {
  SlabSel s;
  s.active = slab >= 0;
  s.last = last != 0;
  s.done = s.active ? done : nullptr;
  s.lo = s.active ? hdr->slab_lo[slot][slab] : 0u;
  s.hi = (s.active && !s.last) ? hdr->slab_lo[slot][slab + 1] : 0xffffffffu;
  return s;
}

// The rectangle Gaussian i is binned with in this call (empty if it is not).
__device__ __forceinline__ ushort4 slab_rect(const ushort4* __restrict__ rects, const uint32_t* __restrict__ depth,
                                             int64_t i, int64_t hi, const SlabSel& sel, int gx) {
  const ushort4 none = make_ushort4(0, 0, 0, 0);
  if (i >= hi) return none;
  const ushort4 r = rects[i];
  if (!sel.active || r.z <= r.x) return r;
  const uint32_t d = depth[i];
  if (d < sel.lo || (!sel.last && d >= sel.hi)) return none;
  if (sel.done) {
    bool open = false;
    for (int ty = r.y; ty < r.w && !open; ++ty)
      for (int tx = r.x; tx < r.z; ++tx)
        if (!sel.done[ty * gx + tx]) { open = true; break; }
    if (!open) return none;
  }
  return r;
}

struct LocalBox {
  int x0, y0, w, h;
  bool ok;
  __device__ __forceinline__ int idx(int tx, int ty) const { return (ty - y0) * w + (tx - x0); }
};

__device__ __forceinline__ bool big(const ushort4& r) { return (r.z - r.x) * (r.w - r.y) > kBigRect; }

// Warp-cooperative expansion of the (Gaussian, tile) items of the 32
// Gaussians held by the lanes (lane l holds rectangle r): the items are
// numbered by an exclusive scan of the rectangle areas and dealt out 32 at a
// time, one per lane, so every lane works on one item per round whatever the
// rectangle sizes.  f(src_lane, tx, ty) is called for each item.
// q = local / w for 0 <= local < 2^22, 1 <= w: (local + 0.5) / w lies at
// least 0.5 / w away from an integer, far more than the error of the
// approximate quotient, so truncation gives the exact integer quotient.
__device__ __forceinline__ int div_small(int local, int w) {
  return local < (1 << 22) ? (int)__fdividef((float)local + 0.5f, (float)w) : local / w;
}

template <typename F>
__device__ __forceinline__ void expand_items(const ushort4& r, F&& f) {
  const int lane = threadIdx.x & 31;
  const int w = r.z > r.x ? r.z - r.x : 0, h = r.w > r.y ? r.w - r.y : 0;
  const int c = w * h;
  int incl = c;
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, off);
    if (lane >= off) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - c;
  const int packed = (int)r.x | ((int)r.y << 16);
  for (int k0 = 0; k0 < total; k0 += 32) {
    const int item = k0 + lane;
    int src = 0;  // largest lane whose first item is <= item (it owns the item)
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      const int e = __shfl_sync(kFull, excl, src + step);
      if (e <= item) src += step;
    }
    const int e_src = __shfl_sync(kFull, excl, src);
    const int w_src = __shfl_sync(kFull, w, src);
    const int p_src = __shfl_sync(kFull, packed, src);
    if (item < total) {
      const int local = item - e_src;
      const int yy = div_small(local, w_src);
      f(src, (p_src & 0xffff) + (local - yy * w_src), (p_src >> 16) + yy);
    }
  }
}

// Block-wide bounding box of the chunk's non-big rectangles (one per thread).
__device__ LocalBox chunk_box(const ushort4& r) {
  __shared__ int s_box[4];
  if (threadIdx.x == 0) { s_box[0] = 1 << 30; s_box[1] = 1 << 30; s_box[2] = 0; s_box[3] = 0; }
  __syncthreads();
  int x0 = 1 << 30, y0 = 1 << 30, x1 = 0, y1 = 0;
  if (r.z > r.x && !big(r)) {
    x0 = r.x; y0 = r.y; x1 = r.z; y1 = r.w;
  }
  for (int off = 16; off > 0; off >>= 1) {
    x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, off));
    y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, off));
    x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, off));
    y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&s_box[0], x0); atomicMin(&s_box[1], y0); atomicMax(&s_box[2], x1); atomicMax(&s_box[3], y1);
  }
  __syncthreads();
  LocalBox b;
  b.x0 = s_box[0];
  b.y0 = s_box[1];
  b.w = max(0, s_box[2] - s_box[0]);
  b.h = max(0, s_box[3] - s_box[1]);
  b.ok = (b.w + 1) * (b.h + 1) <= kLocalMax;  // the counting pass's difference array has one more row and column
  __syncthreads();
  return b;
}

static_assert(kChunk == kBinThreads, "one Gaussian per binning thread");

__global__ void __launch_bounds__(kBinThreads) count_kernel(const ushort4* __restrict__ rects,
                                                            const uint32_t* __restrict__ depth, int64_t n,
                                                            int gx, uint32_t* __restrict__ tile_count,
                                                            uint32_t* __restrict__ tile_glob,
                                                            uint32_t* __restrict__ run_base,
                                                            const WsHeader* __restrict__ hdr, int slot, int slab,
                                                            int last, const uint8_t* __restrict__ done) {
  __shared__ uint32_t s_cnt[kLocalMax];
  const SlabSel sel = slab_sel(hdr, slot, slab, last, done);
  const int64_t lo = blockIdx.x * kChunk, hi = min(n, lo + kChunk);
  const ushort4 r = slab_rect(rects, depth, lo + threadIdx.x, hi, sel, gx);
  const LocalBox box = chunk_box(r);
  const int area = box.w * box.h;
  // Per-tile counts of the chunk's box from a 2D difference array: each
  // rectangle adds +1 / -1 / -1 / +1 at its four corners of a (w + 1) x
  // (h + 1) grid, and prefix sums along x then y give, at every tile, the
  // number of rectangles covering it (items in done tiles are counted here
  // but neither reserved nor filled).  Big rectangles, and every rectangle
  // of a chunk whose box is too large, count item by item in global memory.
  const int pw = box.w + 1;
  if (box.ok)
    for (int t = threadIdx.x; t < pw * (box.h + 1); t += blockDim.x) s_cnt[t] = 0u;
  __syncthreads();
  const bool local = box.ok && r.z > r.x && !big(r);
  if (local) {
    const int x0 = r.x - box.x0, x1 = r.z - box.x0, y0 = r.y - box.y0, y1 = r.w - box.y0;
    atomicAdd(&s_cnt[y0 * pw + x0], 1u);
    atomicAdd(&s_cnt[y0 * pw + x1], 0xffffffffu);
    atomicAdd(&s_cnt[y1 * pw + x0], 0xffffffffu);
    atomicAdd(&s_cnt[y1 * pw + x1], 1u);
  }
  {
    const ushort4 rg = local ? make_ushort4(0, 0, 0, 0) : r;
    expand_items(rg, [&](int src, int tx, int ty) {
      if (sel.skip_tile(ty * gx + tx)) return;
      atomicAdd(&tile_glob[ty * gx + tx], 1u);
    });
  }
  __syncthreads();
  if (box.ok) {
    for (int y = threadIdx.x; y < box.h; y += blockDim.x) {  // along x, one row per thread
      uint32_t run = 0u;
      for (int x = 0; x < box.w; ++x) { run += s_cnt[y * pw + x]; s_cnt[y * pw + x] = run; }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < box.w; x += blockDim.x) {  // along y, one column per thread
      uint32_t run = 0u;
      for (int y = 0; y < box.h; ++y) { run += s_cnt[y * pw + x]; s_cnt[y * pw + x] = run; }
    }
  }
  __syncthreads();
  // reserve this CTA's run in every tile of its box (offset inside the tile's list)
  if (box.ok) {
    uint32_t* base = run_base + (int64_t)blockIdx.x * kLocalMax;
    for (int t = threadIdx.x; t < area; t += blockDim.x) {
      const int ty = t / box.w, tx = t - ty * box.w;
      const uint32_t c = s_cnt[ty * pw + tx];
      const int g = (box.y0 + ty) * gx + box.x0 + tx;
      base[t] = (c && !sel.skip_tile(g)) ? atomicAdd(&tile_count[g], c) : 0u;
    }
  }
}

// Exclusive scan of the tile counts (reserved runs + big-rectangle items; one
// CTA), capacity check; the fill cursor of a tile starts after its reserved
// runs; the counters are reset for the next view.
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* __restrict__ tile_count,
                                                    uint32_t* __restrict__ tile_glob,
                                                    uint32_t* __restrict__ tile_start,
                                                    uint32_t* __restrict__ tile_fill, int ntiles,
                                                    int64_t capacity, WsHeader* __restrict__ hdr,
                                                    int slot) {
  __shared__ uint32_t s_warp[32];
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    const int t = base + threadIdx.x;
    const uint32_t local = t < ntiles ? tile_count[t] : 0u;
    uint32_t v = t < ntiles ? local + tile_glob[t] : 0u;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const unsigned long long carry = s_carry;
    const uint32_t excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0u);
    if (t < ntiles) {
      tile_start[t] = (uint32_t)(carry + excl);
      tile_count[t] = 0u;
      tile_glob[t] = 0u;
      tile_fill[t] = local;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = carry + excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // the other depth-range slot is next written by the following view's projection
    hdr->drange[slot ^ 1][0] = 0xffffffffu;
    hdr->drange[slot ^ 1][1] = 0u;
    const unsigned long long total = s_carry;
    tile_start[ntiles] = (uint32_t)total;
    if ((long long)total > capacity || total > 0xffffffffull) atomicOr(&hdr->status, kStatCapacity);
    atomicAdd(&hdr->listed, total);
    atomicMax(&hdr->max_dups_view, (int)min(total, 0x7fffffffull));
  }
}

__global__ void __launch_bounds__(kBinThreads) fill_kernel(
    const ushort4* __restrict__ rects, const uint32_t* __restrict__ depth, const int32_t* __restrict__ orig,
    int64_t n, int gx, const uint32_t* __restrict__ tile_start, uint32_t* __restrict__ tile_fill,
    const uint32_t* __restrict__ run_base, unsigned long long* __restrict__ keys, const WsHeader* __restrict__ hdr,
    int slot, int slab, int last, const uint8_t* __restrict__ done) {
  __shared__ uint32_t s_cnt[kLocalMax];
  __shared__ uint32_t s_base[kLocalMax];
  if (hdr->status & kStatCapacity) return;
  const SlabSel sel = slab_sel(hdr, slot, slab, last, done);
  const int64_t lo = blockIdx.x * kChunk, hi = min(n, lo + kChunk);
  const ushort4 r = slab_rect(rects, depth, lo + threadIdx.x, hi, sel, gx);
  const LocalBox box = chunk_box(r);
  const int area = box.w * box.h;
  if (box.ok) {
    // the runs reserved by the counting pass (same chunk, same box)
    const uint32_t* base = run_base + (int64_t)blockIdx.x * kLocalMax;
    for (int t = threadIdx.x; t < area; t += blockDim.x) {
      s_base[t] = tile_start[(box.y0 + t / box.w) * gx + box.x0 + t % box.w] + base[t];
      s_cnt[t] = 0u;
    }
    __syncthreads();
  }
  {
    const int64_t i = lo + threadIdx.x;
    const unsigned long long my_key =
        i < hi ? (((unsigned long long)depth[i] << 32) | (uint32_t)orig[i]) : 0ull;
    const unsigned lmask = __ballot_sync(kFull, box.ok && !big(r));
    // the key of the owning lane is fetched for every round (all lanes shuffle)
    const int lane = threadIdx.x & 31;
    const int w = r.z > r.x ? r.z - r.x : 0, h = r.w > r.y ? r.w - r.y : 0;
    const int c = w * h;
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, off);
      if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - c;
    const int packed = (int)r.x | ((int)r.y << 16);
    // A warp whose Gaussians all take the chunk-local path and whose
    // rectangles overlap enough walks the union of its rectangles tile by
    // tile instead: the lanes covering a tile take consecutive slots of its
    // run (one shared atomic per warp and tile) and write their keys with one
    // coalesced store.  The slots reserved per tile are the items the
    // item-by-item path would add, so both paths fill the same runs.
    const bool mine = r.z > r.x && r.w > r.y;
    const bool all_local = (lmask | ~__ballot_sync(kFull, mine)) == kFull;
    const int ux0 = __reduce_min_sync(kFull, mine ? (int)r.x : 0x7fffffff);
    const int uy0 = __reduce_min_sync(kFull, mine ? (int)r.y : 0x7fffffff);
    const int ux1 = __reduce_max_sync(kFull, mine ? (int)r.z : 0);
    const int uy1 = __reduce_max_sync(kFull, mine ? (int)r.w : 0);
    const int uarea = (ux1 > ux0 && uy1 > uy0) ? (ux1 - ux0) * (uy1 - uy0) : 0;
    if (all_local && total > 0 && uarea * kUnionItemsPerTile <= total) {
      const unsigned lt = (1u << lane) - 1u;
      for (int ty = uy0; ty < uy1; ++ty) {
        const bool row_in = mine && ty >= (int)r.y && ty < (int)r.w;
        if (!__any_sync(kFull, row_in)) continue;
        for (int tx = ux0; tx < ux1; ++tx) {
          const bool in = row_in && tx >= (int)r.x && tx < (int)r.z;
          const unsigned m = __ballot_sync(kFull, in);
          if (m == 0u || sel.skip_tile(ty * gx + tx)) continue;
          const int t = box.idx(tx, ty);
          const int leader = __ffs(m) - 1;
          uint32_t b0 = 0u;
          if (lane == leader) b0 = atomicAdd(&s_cnt[t], (uint32_t)__popc(m));
          b0 = __shfl_sync(kFull, b0, leader);
          if (in) keys[s_base[t] + b0 + __popc(m & lt)] = my_key;
        }
      }
    } else
    for (int k0 = 0; k0 < total; k0 += 32) {
      const int item = k0 + lane;
      int src = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int e = __shfl_sync(kFull, excl, src + step);
        if (e <= item) src += step;
      }
      const int e_src = __shfl_sync(kFull, excl, src);
      const int w_src = __shfl_sync(kFull, w, src);
      const int p_src = __shfl_sync(kFull, packed, src);
      const unsigned long long key = __shfl_sync(kFull, my_key, src);
      if (item < total) {
        const int local = item - e_src;
        const int yy = div_small(local, w_src);
        const int tx = (p_src & 0xffff) + (local - yy * w_src), ty = (p_src >> 16) + yy;
        if (sel.skip_tile(ty * gx + tx)) continue;
        uint32_t pos;
        if ((lmask >> src) & 1u) {
          const int t = box.idx(tx, ty);
          pos = s_base[t] + atomicAdd(&s_cnt[t], 1u);
        } else {
          const int t = ty * gx + tx;
          pos = tile_start[t] + atomicAdd(&tile_fill[t], 1u);
        }
        keys[pos] = key;
      }
    }
  }
}

}  // namespace

size_t binning_run_base_bytes(int64_t n) {
  return sizeof(uint32_t) * (size_t)((n + kChunk - 1) / kChunk) * (size_t)kLocalMax;
}

cudaError_t launch_binning(const CamArgs& cam, int64_t n, const UpliftWs& ws, int slot,
                           cudaStream_t st, int slab, bool last_slab) {
  const int ntiles = cam.gx * cam.gy;
  const int blocks = (int)((n + kChunk - 1) / kChunk);
  const uint8_t* done = slab > 0 ? ws.tile_done : nullptr;
  const int last = last_slab ? 1 : 0;
  if (n > 0)
    count_kernel<<<blocks, kBinThreads, 0, st>>>(ws.rect, ws.depth, n, cam.gx, ws.tile_count, ws.tile_glob,
                                                 ws.run_base, ws.hdr, slot, slab, last, done);
  scan_kernel<<<1, 1024, 0, st>>>(ws.tile_count, ws.tile_glob, ws.tile_start, ws.tile_fill, ntiles,
                                  ws.dup_capacity, ws.hdr, slot);
  if (n > 0)
    fill_kernel<<<blocks, kBinThreads, 0, st>>>(ws.rect, ws.depth, ws.sp.orig, n, cam.gx, ws.tile_start,
                                                ws.tile_fill, ws.run_base, ws.keys, ws.hdr, slot, slab, last,
                                                done);
  g_launches += n > 0 ? 3 : 1;
  return cudaGetLastError();
}

}  // namespace scoup
