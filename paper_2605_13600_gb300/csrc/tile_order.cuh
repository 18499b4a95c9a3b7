// tile_order.cuh -- front-to-back ordering of one tile's key list, window by
// window, for a whole CTA (used by the render and render-backward kernels).
//
// Keys are (depth bits << 32 | original Gaussian index), unique per tile.  A
// histogram over kNB buckets (a monotone map of the depth bits onto the
// view's depth range) is built once; each window is a run of whole buckets
// holding at most kWin keys, gathered by a counting sort by bucket and then
// ordered exactly by rank inside each bucket.  A bucket with more than kWin
// keys is consumed in sub-windows found by a block-wide radix select.
#pragma once

#include "scoup_internal.cuh"

namespace scoup {

// Key loads a thread keeps in flight in the list passes (kLB, a template
// parameter of order_init and order_next_window): 4 by default, more where
// registers allow.
constexpr int kLoadBatch = 4;

// kSync_: 0 when the whole CTA orders (the functions below synchronise with
// __syncthreads and stride by blockDim.x); otherwise the number of threads,
// the CTA's first kSync_, that order on named barrier 1 while the rest of the
// CTA does other work.
template <int kWin_, int kLogNB_, int kSync_ = 0>
struct OrderSmem {
  static constexpr int kWin = kWin_;
  static constexpr int kNB = 1 << kLogNB_;
  static constexpr int kLogNB = kLogNB_;
  static constexpr int kSync = kSync_;
  __device__ static __forceinline__ int nthreads() { return kSync ? kSync : (int)blockDim.x; }
  __device__ static __forceinline__ void sync() {
    if constexpr (kSync > 0) asm volatile("bar.sync 1, %0;" ::"n"(kSync) : "memory");
    else __syncthreads();
  }
  uint32_t bstart[kNB + 1];
  uint32_t bcur[kNB];
  unsigned long long win[kWin];
  uint32_t hist[256];
  unsigned long long red_min, red_max;
  unsigned int cursor;
  int sel_digit, sel_rank, win_b1;
};

struct OrderBuckets {
  uint32_t dmin;
  int shift;
  int nb;
  // monotone in the key and always inside [0, nb)
  __device__ __forceinline__ int operator()(unsigned long long key) const {
    const uint32_t d = (uint32_t)(key >> 32);
    return (int)min((d > dmin ? d - dmin : 0u) >> shift, (uint32_t)(nb - 1));
  }
};

struct OrderState {
  int b0 = 0;
  bool in_split = false, split_first = true;
  unsigned long long split_last = 0ull;
  int consumed = 0;
};

template <class S>
__device__ OrderBuckets order_buckets(const WsHeader* hdr, int slot) {
  OrderBuckets bk;
  const uint32_t dmin = hdr->drange[slot][0], dmax = hdr->drange[slot][1];
  const uint32_t span = dmax >= dmin ? dmax - dmin : 0u;
  const int nb = span ? 32 - __clz((int)span) : 0;
  bk.dmin = dmin;
  bk.shift = nb > S::kLogNB ? nb - S::kLogNB : 0;
  bk.nb = S::kNB;
  return bk;
}

// Histogram + exclusive scan into sm.bstart (S::nthreads() threads, a
// multiple of 32 dividing kNB).
template <class S, int kLB = kLoadBatch>
__device__ void order_init(S& sm, const unsigned long long* __restrict__ keys, int n, const OrderBuckets& bk) {
  const int tid = threadIdx.x, nt = S::nthreads(), lane = tid & 31, warp = tid >> 5;
  for (int b = tid; b < S::kNB; b += nt) sm.bcur[b] = 0u;
  S::sync();
  // kLB keys per thread are loaded before their atomics, so each
  // thread has that many global loads in flight at once
  for (int i0 = tid; i0 < n; i0 += kLB * nt) {
    unsigned long long kk[kLB];
#pragma unroll
    for (int u = 0; u < kLB; ++u) {
      const int i = i0 + u * nt;
      kk[u] = i < n ? keys[i] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kLB; ++u)
      if (i0 + u * nt < n) atomicAdd(&sm.bcur[bk(kk[u])], 1u);
  }
  S::sync();
  const int per = S::kNB / nt;
  uint32_t sum = 0;
  for (int q = 0; q < per; ++q) sum += sm.bcur[tid * per + q];
  uint32_t incl = sum;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) sm.hist[warp] = incl;
  S::sync();
  uint32_t run = incl - sum;
  for (int w = 0; w < warp; ++w) run += sm.hist[w];
  for (int q = 0; q < per; ++q) {
    const uint32_t c = sm.bcur[tid * per + q];
    sm.bstart[tid * per + q] = run;
    run += c;
  }
  if (tid == nt - 1) sm.bstart[S::kNB] = run;
  S::sync();
}

// The rank-th smallest (0-based) key in bucket b with (first || key > last).
template <class S>
__device__ unsigned long long order_select(S& sm, const unsigned long long* __restrict__ keys, int n,
                                           const OrderBuckets& bk, int b, unsigned long long last,
                                           bool first, int rank) {
  const int tid = threadIdx.x, nt = S::nthreads();
  if (tid == 0) { sm.red_min = ~0ull; sm.red_max = 0ull; }
  S::sync();
  unsigned long long lmin = ~0ull, lmax = 0ull;
  for (int i = tid; i < n; i += nt) {
    const unsigned long long k = keys[i];
    if (bk(k) == b && (first || k > last)) { lmin = min(lmin, k); lmax = max(lmax, k); }
  }
  for (int off = 16; off > 0; off >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, off));
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
  }
  if ((tid & 31) == 0) { atomicMin(&sm.red_min, lmin); atomicMax(&sm.red_max, lmax); }
  S::sync();
  const unsigned long long base = sm.red_min, span = sm.red_max - sm.red_min;
  const int nbits = span ? 64 - __clzll((long long)span) : 1;
  unsigned long long prefix = 0ull, pmask = 0ull;
  for (int shift = ((nbits - 1) / 8) * 8; shift >= 0; shift -= 8) {
    for (int d = tid; d < 256; d += nt) sm.hist[d] = 0u;
    S::sync();
    for (int i = tid; i < n; i += nt) {
      const unsigned long long k = keys[i];
      if (bk(k) == b && (first || k > last)) {
        const unsigned long long x = k - base;
        if ((x & pmask) == prefix) atomicAdd(&sm.hist[(x >> shift) & 255u], 1u);
      }
    }
    S::sync();
    if (tid < 32) {
      uint32_t c[8], sum = 0;
      for (int d = 0; d < 8; ++d) { c[d] = sm.hist[tid * 8 + d]; sum += c[d]; }
      uint32_t incl = sum;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
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
    S::sync();
    prefix |= (unsigned long long)sm.sel_digit << shift;
    pmask |= 0xffull << shift;
    rank = sm.sel_rank;
    S::sync();
  }
  return base + prefix;
}

// Next window, sorted front to back into sm.win[0..m).  Returns m, or 0 when
// the list is exhausted, or -1 on an internal inconsistency (status set).
// Block-uniform; every thread of the CTA must call it.
template <class S, int kLB = kLoadBatch>
__device__ int order_next_window(S& sm, const unsigned long long* __restrict__ keys, int n,
                                 const OrderBuckets& bk, OrderState& st, WsHeader* hdr) {
  const int tid = threadIdx.x, nt = S::nthreads();
  constexpr int kWin = S::kWin, kNB = S::kNB;
  // the in-place permutation below reads a whole window before writing it
  if (kWin > 4 * nt) {
    if (tid == 0) atomicOr(&hdr->status, kStatDeviceCheck);
    return -1;
  }
  // skip empty buckets
  while (!st.in_split && st.b0 < kNB && sm.bstart[st.b0 + 1] == sm.bstart[st.b0]) {
    if (tid == 0) {
      const uint32_t base = sm.bstart[st.b0];
      int lo = st.b0 + 1, hi = kNB;  // first bucket >= lo holding a key
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sm.bstart[mid + 1] > base) hi = mid; else lo = mid + 1;
      }
      sm.win_b1 = lo;
    }
    S::sync();
    st.b0 = sm.win_b1;
    S::sync();
  }
  if (st.b0 >= kNB) return 0;
  const uint32_t base = sm.bstart[st.b0];
  const int total_b0 = (int)(sm.bstart[st.b0 + 1] - base);
  if (!st.in_split) {
    if (tid == 0) {
      int lo = st.b0 + 1, hi = kNB;  // largest b1 with bstart[b1] - base <= kWin, or b0 if oversize
      if (sm.bstart[lo] - base > (uint32_t)kWin) {
        sm.win_b1 = st.b0;
      } else {
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sm.bstart[mid] - base <= (uint32_t)kWin) lo = mid; else hi = mid - 1;
        }
        sm.win_b1 = lo;
      }
    }
    S::sync();
  }
  const int b1 = sm.win_b1;
  int m;
  if (!st.in_split && b1 > st.b0) {
    m = (int)(sm.bstart[b1] - base);
    for (int b = st.b0 + tid; b < b1; b += nt) sm.bcur[b] = sm.bstart[b] - base;
    S::sync();
    for (int i0 = tid; i0 < n; i0 += kLB * nt) {
      unsigned long long kk[kLB];
#pragma unroll
      for (int u = 0; u < kLB; ++u) {
        const int i = i0 + u * nt;
        kk[u] = i < n ? keys[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < kLB; ++u) {
        const int b = bk(kk[u]);
        if (i0 + u * nt < n && b >= st.b0 && b < b1) {
          const uint32_t pos = atomicAdd(&sm.bcur[b], 1u);
          if (pos < (uint32_t)kWin) sm.win[pos] = kk[u];
        }
      }
    }
    S::sync();
    // rank inside the bucket, then permute in place (m <= kWin <= 4 nt: one pass)
    for (int p0 = 0; p0 < m; p0 += nt * 4) {
      unsigned long long kk[4];
      int dst[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = p0 + tid + u * nt;
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
      S::sync();
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (dst[u] >= 0) sm.win[dst[u]] = kk[u];
      S::sync();
    }
  } else {
    if (!st.in_split) { st.in_split = true; st.split_first = true; st.consumed = 0; }
    if (tid == 0) atomicAdd(&hdr->split_windows, 1ull);
    const int left = total_b0 - st.consumed;
    unsigned long long hi_key = ~0ull;
    if (left > kWin) hi_key = order_select(sm, keys, n, bk, st.b0, st.split_last, st.split_first, kWin - 1);
    if (tid == 0) sm.cursor = 0u;
    S::sync();
    for (int i = tid; i < n; i += nt) {
      const unsigned long long k = keys[i];
      if (bk(k) == st.b0 && (st.split_first || k > st.split_last) && k <= hi_key) {
        const unsigned pos = atomicAdd(&sm.cursor, 1u);
        if (pos < (unsigned)kWin) sm.win[pos] = k;
      }
    }
    S::sync();
    m = (int)min(sm.cursor, (unsigned)kWin);
    for (int p0 = 0; p0 < m; p0 += nt * 4) {
      unsigned long long kk[4];
      int dst[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = p0 + tid + u * nt;
        dst[u] = -1;
        if (p < m) {
          const unsigned long long k = sm.win[p];
          int r = 0;
          for (int q = 0; q < m; ++q) r += sm.win[q] < k;
          kk[u] = k;
          dst[u] = r;
        }
      }
      S::sync();
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (dst[u] >= 0) sm.win[dst[u]] = kk[u];
      S::sync();
    }
  }
  S::sync();
  if (m <= 0) {
    if (tid == 0) atomicOr(&hdr->status, kStatDeviceCheck);
    return -1;
  }
  // advance
  if (st.in_split) {
    st.consumed += m;
    st.split_last = sm.win[m - 1];
    st.split_first = false;
    if (st.consumed >= total_b0) { st.in_split = false; st.b0 += 1; }
  } else {
    st.b0 = b1;
  }
  return m;
}

}  // namespace scoup
