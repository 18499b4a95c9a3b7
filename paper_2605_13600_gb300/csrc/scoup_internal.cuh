// scoup_internal.cuh -- shared definitions of the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/scoup.h"
#include "../../include/scoup_selftest.h"

#include <atomic>

namespace scoup {

// Kernel launches issued by the library (every launcher adds its count).
extern std::atomic<long long> g_launches;

// Streaming multiprocessors of the current device (queried once per device);
// grid sizes of the grid-stride kernels are multiples of it.
int num_sms();

constexpr int kTile = 16;            // 16x16 pixel tiles define binning membership (3DGS)
constexpr int kTilePixels = kTile * kTile;

// Device status bits (workspace header).
constexpr int kStatCapacity = 1;
constexpr int kStatDeviceCheck = 2;
constexpr int kStatTimeout = 4;

// Depth slabs.  The visible Gaussians of a view are split by depth into up to
// kMaxSlabs slabs (front to back) at quantiles of their depth; every key of
// slab s is smaller than every key of slab s + 1, so compositing the slabs in
// turn, each in exact (depth, index) order, is compositing the whole list in
// that order.  Slab s > 0 is binned only into tiles with a pixel that is still
// open, which skips the Gaussians hidden behind saturated tiles.
constexpr int kMaxSlabs = 6;
constexpr int kDepthBuckets = 2048;        // depth histogram: float bits >> 16, from 0.2 up
constexpr uint32_t kDepthBucketBase = 0x3E4Cu;  // (bits of 0.2f) >> 16

// Workspace header: status word, per-view depth range (double-buffered by
// view parity in each of the two view pipelines), scene bounding box,
// counters and the slab bounds of each slot, 256 bytes.
struct WsHeader {
  int32_t status;
  int32_t max_dups_view;
  uint32_t drange[4][2];  // [2 lane + (view & 1)] = {min, max} float bits of visible depths
  uint32_t bbox[3][2];    // order-preserving bits of the means' bounding box
  unsigned long long visible;
  unsigned long long duplicates;
  unsigned long long evaluated;
  unsigned long long contributions;
  unsigned long long flushes;
  unsigned long long atomics;
  unsigned long long listed;
  uint32_t slab_lo[4][kMaxSlabs];  // [slot][s]: smallest depth bits of slab s (slab 0 starts at 0)
  uint32_t pp_blocks[4];           // projection CTAs finished in this slot's view (last one sets slab_lo)
  unsigned long long split_windows;  // windows cut out of a depth bucket holding more than a window
  unsigned long long reserved[2];
};
static_assert(sizeof(WsHeader) == 256, "header size");

// Slab schedule of one uplift: nslabs slabs whose bounds sit at the given
// quantiles of the visible Gaussians' depths (nslabs - 1 of them, ascending).
struct SlabPlan {
  int nslabs;
  float q[kMaxSlabs - 1];
};

// Projected Gaussian of one view, 32 bytes:
//   a = (mx, my, qa, qb), b = (qc, opacity, tau, log2(opacity))
// power(dx, dy) = dx*(qa*dx + qb*dy) + (qc*dy)*dy and the Gaussian is
// accepted at a pixel iff tau <= power <= 0  (tau: smallest float with
// o*exp(tau) >= 1/255).
struct __align__(16) ProjRec {
  float4 a;
  float4 b;
};

// Conservative test: can any pixel centre of the box [x0, x0+w-1] x
// [y0, y0+h-1] reach power >= tau for this record?  The maximum of the concave
// exponent over the box is at the clamped centre or on one of the four edges
// (each a 1D concave quadratic with its vertex clamped to the edge); the box
// is rejected only if that maximum is below tau by a margin far above the
// binary32 rounding of either evaluation, so a rejected box holds no pixel
// that passes the per-pixel alpha test.
__device__ __forceinline__ bool box_may_hit(const ProjRec& r, float x0, float y0, float w, float h) {
  const float mx = r.a.x, my = r.a.y, qa = r.a.z, qb = r.a.w, qc = r.b.x, tau = r.b.z;
  if (!(qa < 0.0f && qc < 0.0f)) return true;
  const float x1 = x0 + (w - 1.0f), y1 = y0 + (h - 1.0f);
  if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
  // argmax over dy along an edge x = const (dy = kx * dx) and over dx along an
  // edge y = const (dx = ky * dy); an approximate quotient only moves the
  // evaluation point slightly on a flat maximum, far inside the margin below
  const float kx = __fdividef(-qb, 2.0f * qc);
  const float ky = __fdividef(-qb, 2.0f * qa);
  float best = -INFINITY;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dx = mx - (e ? x1 : x0);
    const float dy = my - fminf(y1, fmaxf(y0, my - kx * dx));
    best = fmaxf(best, qa * dx * dx + qb * dx * dy + qc * dy * dy);
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dy = my - (e ? y1 : y0);
    const float dx = mx - fminf(x1, fmaxf(x0, mx - ky * dy));
    best = fmaxf(best, qa * dx * dx + qb * dx * dy + qc * dy * dy);
  }
  return best >= tau - (0.01f + 1e-3f * fabsf(best));
}

// Conservative test of a whole grid of boxes at once: bit r * kCols + c is
// set when box (c, r) -- pixels x0 + c w .. x0 + c w + w - 1 by
// y0 + r h .. y0 + r h + h - 1 -- may hold a pixel centre with power >= tau.
// In offsets (u, v) = (x - mx, y - my) the accepted set is the ellipse
// E = {qa u^2 + qb u v + qc v^2 >= lvl}, with the level lvl a margin below
// tau that covers the binary32 rounding of the per-pixel exponent (the terms
// of the exponent reach |tau| times the ellipse's aspect ratio, so the margin
// grows with it).  For each row of boxes (a strip va <= v <= vb) the x-extent
// of E inside the strip is found in closed form: the right end of E's chord
// at height v is a concave function of v whose maximum is E's rightmost point
// (u_e, v_e), so over the strip it peaks at v = clamp(v_e, va, vb); the left
// end, by symmetry, at clamp(-v_e, va, vb).  A strip that misses E has no
// chord there (negative discriminant).  The extent is widened by 0.01 px.
template <int kCols, int kRows>
__device__ __forceinline__ uint32_t box_grid_mask(const ProjRec& r, float x0, float y0, float w, float h) {
  constexpr uint32_t kAll = kCols * kRows >= 32 ? 0xffffffffu : ((1u << (kCols * kRows)) - 1u);
  const float mx = r.a.x, my = r.a.y, qa = r.a.z, qb = r.a.w, qc = r.b.x, tau = r.b.z;
  const float det = 4.0f * qa * qc - qb * qb;  // > 0 for a negative-definite exponent
  if (!(qa < 0.0f && qc < 0.0f && det > 0.0f && tau < 0.0f)) return kAll;
  const float aspect = 4.0f * (qa + qc) * (qa + qc) / det;  // >= the ratio of the ellipse's axes squared
  const float lvl = tau - (0.02f + 2e-3f * fabsf(tau) + 1e-5f * fabsf(tau) * aspect);
  const float c4 = 4.0f * qa * lvl;                           // > 0
  const float ue = sqrtf(4.0f * qc * lvl / det);              // rightmost point of E
  const float ve = -qb * ue / (2.0f * qc);
  const float inv2a = 0.5f / qa;                              // < 0
  uint32_t mask = 0u;
#pragma unroll
  for (int row = 0; row < kRows; ++row) {
    const float va = y0 + (float)row * h - my - 0.01f, vb = va + (h - 1.0f) + 0.02f;
    const float vr = fminf(fmaxf(ve, va), vb), vl = fminf(fmaxf(-ve, va), vb);
    const float dr = fmaf(-det, vr * vr, c4), dl = fmaf(-det, vl * vl, c4);
    if (dr < 0.0f && dl < 0.0f) continue;
    // chord roots (-qb v -/+ sqrt(D)) / (2 qa): the right end takes -sqrt(D)
    const float xr = mx + (-qb * vr - sqrtf(fmaxf(dr, 0.0f))) * inv2a + 0.01f;
    const float xl = mx + (-qb * vl + sqrtf(fmaxf(dl, 0.0f))) * inv2a - 0.01f;
#pragma unroll
    for (int col = 0; col < kCols; ++col) {
      const float bx0 = x0 + (float)col * w;
      if (xr >= bx0 && xl <= bx0 + (w - 1.0f)) mask |= 1u << (row * kCols + col);
    }
  }
  return mask;
}

// One relevancy term of App. B, Eq. 9: e^{a s_q} / (e^{a s_q} + e^{a s_k}) =
// 1 / (1 + e^{a (s_k - s_q)}), with s_k the largest canonical similarity (the
// term decreases in s_k, so it is the minimum over the canonical phrases).
// The exponential is the SFU's base-2 one and the quotient the fast
// reciprocal (about 2^-21 relative together); both relevancy paths use this
// one function, so they agree bit for bit.
__device__ __forceinline__ float relevancy_term(float alpha, float s_canon_max, float s_query) {
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(alpha * 1.4426950408889634f * (s_canon_max - s_query)));
  return fminf(1.0f, __fdividef(1.0f, 1.0f + e));
}

// Region maps and code tables of one view, one per semantic level (a single
// level for scoup_uplift; up to three for scoup_uplift_levels).
constexpr int kMaxLevels = 3;
struct LevelCodes {
  const int32_t* rmap[kMaxLevels];  // this view's region map of each level
  const int32_t* ci[kMaxLevels];    // code tables [R, s] of each level
  const float* cv[kMaxLevels];
  int s[kMaxLevels];
  int R[kMaxLevels];
  int L;      // number of levels
  int s_tot;  // sum of s over the levels (entries of a combined region code)
};

struct CamArgs {
  float vm[12];
  float fx, fy, cx, cy;
  int width, height;
  int gx, gy;  // tile grid
};

// One view of a batched chunk, as the drain kernel takes it: the arguments
// of the per-view tile kernel (single level, one slab) and the view's tiles.
struct TileJob {
  CamArgs cam;
  LevelCodes lc;
  const ProjRec* proj;
  const unsigned long long* keys;
  const uint32_t* tile_start;
  float* accum;
  float* comp;                 // compensation array (compensated form) or null
  WsHeader* hdr;        // the view's own header: depth range, counters, status
  WsHeader* scene_hdr;  // the scene's header, into which the view's counters are merged
  int slot;                    // depth-range slot of the view in its own header
  int C;
  int tiles;
  int scene;
};

// Scene copy in spatial (Morton) order; orig[p] is the caller's index.
struct SceneP {
  float* means;    // [n,3]
  float* scales;   // [n,3]
  float* quats;    // [n,4], 16-byte aligned
  float* opacity;  // [n]
  float* tau;      // [n] alpha-threshold exponent
  int32_t* orig;   // [n]
};

// Workspace carve-up for one uplift call.
struct UpliftWs {
  WsHeader* hdr;
  SceneP sp;
  uint32_t* cell;           // [n] Morton cell of each Gaussian
  uint32_t* cells_scratch;  // counting-sort scratch (reorder_scratch_bytes())
  ProjRec* proj;            // [n] by original index
  uint32_t* depth;          // [n] float bits of camera depth, spatial order
  ushort4* rect;            // [n] listed tiles (x_lo, y_lo, x_hi, y_hi), spatial order: the 3DGS
                            //     rectangle cut to the alpha >= 1/255 ellipse's box; empty if culled
  uint32_t* tile_count;     // [max_tiles + 1] runs reserved per tile (binning)
  uint32_t* tile_glob;      // [max_tiles + 1] big-rectangle items per tile (binning)
  uint32_t* run_base;       // [chunks x box tiles] offset of each binning CTA's run in a tile list
  uint32_t* tile_start;     // [max_tiles + 1]
  uint32_t* tile_fill;      // [max_tiles]
  float* pix_state;         // [max_tiles * 256] per pixel between slabs: 0 = untouched (T = 1),
                            //     > 0 = transmittance T, < 0 = stopped
  uint8_t* tile_done;       // [max_tiles] 1 once every pixel of the tile has stopped
  uint32_t* dhist;          // [kDepthBuckets] depth histogram of the view being projected
  unsigned long long* keys; // [dup_capacity] (depth bits << 32 | gid)
  int64_t dup_capacity;
  int max_tiles;
};

// Records msg as the calling thread's last error and returns code.
int set_error(int code, const char* msg);

// Arguments of one uplift call (the scoup_uplift parameters).
struct UpliftCall {
  const scoup_scene* scene;
  const scoup_camera* cams;
  int32_t V;
  const int32_t* region_maps;
  const int64_t* map_offsets;
  int32_t R_total;
  const int32_t* code_idx;
  const float* code_val;
  int32_t s, C, K;
  float* accum;
  int32_t accum_mode;
  int32_t* topk_idx;
  float* topk_val;
  int32_t L = 0;                        // > 0: semantic levels in `levels` replace the
  const scoup_level* levels = nullptr;  // single-level region map and code fields above
  // region_maps in HOST memory (single level): each view's map is copied into
  // a device ring of kMapStageSlots slots of map_stage_cap entries, on a
  // library copy stream, just ahead of the view's tile kernel
  bool maps_on_host = false;
  int32_t* map_stage = nullptr;
  int64_t map_stage_cap = 0;
};
constexpr int kMapStageSlots = 4;

// Validates and enqueues one uplift on `st` without synchronising; warp_w is
// the tile kernel's warp pixel-block width (8, 16 or 4).  *hdr_out receives
// the workspace header that holds the call's status and counters.
// view_lanes = 2 runs even and odd views in two pipelines (a second stream)
// when the workspace holds both.
int uplift_call(const UpliftCall& c, void* workspace, size_t ws_bytes, int warp_w, const struct WsHeader** hdr_out,
                cudaStream_t st, int view_lanes = 1);
size_t uplift_required_bytes(int64_t n, const scoup_camera* cams, int32_t V, int32_t s, int32_t K, int32_t R_total,
                             int64_t dup_capacity);
int uplift_stats(const struct WsHeader* dev_hdr, scoup_stats* stats, cudaStream_t st);
// Parts of an uplift workspace (api.cu): the scene part (header, Morton-ordered
// scene copy, codes filtered to K entries) and one view part (records, depth,
// rectangles, tile counters, slab state); the carve functions lay a part out
// from a 256-byte aligned base and return its size.
size_t uplift_scene_part_bytes(int64_t n, int64_t code_rows_k);
size_t uplift_view_part_bytes(int64_t n, int max_tiles);
size_t carve_scene_part(void* base, int64_t n, int64_t code_rows_k, UpliftWs* w, int32_t** codes_i,
                        float** codes_v);
size_t carve_view_part(void* base, int64_t n, int max_tiles, UpliftWs* w);
CamArgs camera_args(const scoup_camera& c);
int check_scene_views(const scoup_scene* scene, const scoup_camera* cams, int32_t V, int* max_tiles);
void header_stats(const struct WsHeader& h, scoup_stats* stats);

// Launchers (each defined in its own translation unit).
size_t reorder_scratch_bytes();
cudaError_t launch_reorder(const scoup_scene& sc, const UpliftWs& ws, cudaStream_t st);
// With slabs (plan and plan->nslabs > 1) the projection also clears the
// per-pixel slab state and builds the depth histogram from which its last CTA
// sets hdr->slab_lo[slot].
cudaError_t launch_preprocess(const scoup_scene& sc, const CamArgs& cam, const UpliftWs& ws,
                              int slot, cudaStream_t st, const SlabPlan* plan = nullptr);
size_t binning_run_base_bytes(int64_t n);
// slab < 0: every listed Gaussian into every tile of its rectangle.  slab s >= 0:
// only Gaussians of slab s (bounds in hdr->slab_lo[slot]; s = last takes no
// upper bound), and for s > 0 only into tiles not yet marked done.
cudaError_t launch_binning(const CamArgs& cam, int64_t n, const UpliftWs& ws, int slot,
                           cudaStream_t st, int slab = -1, bool last_slab = true);
// Accumulator rows are Crow = L * C floats wide; level l owns columns [l C, (l + 1) C).
// slab / nslabs: the tiles composite slab `slab` of nslabs, resuming each
// pixel from ws.pix_state unless slab == 0 and saving it unless it is the last.
cudaError_t launch_uplift_tiles(const CamArgs& cam, const UpliftWs& ws, int slot, const LevelCodes& lc, int C,
                                int Crow, float* accum, float* comp, int warp_w, cudaStream_t st,
                                int slab = 0, int nslabs = 1);
// Batched chunk: one persistent launch composites every tile of njobs <=
// kMaxDrainJobs views (HOST jobs[njobs], copied into the launch's parameters).
// tile0[j] is the index of view j's first tile in the chunk's item space
// (tile0[0] = 0, each the sum of the tiles before it); CTAs take items from
// *counter (DEVICE, zero before the launch).
constexpr int kMaxDrainJobs = 64;
cudaError_t launch_uplift_drain(const TileJob* jobs, const uint32_t* tile0, int njobs, unsigned* counter,
                                bool compensated, int warp_w, cudaStream_t st);
size_t render_smem_bytes(int C, int K);
bool render_uses_mma(int C, int K);
bool render_mma_supported(int C, int K);
size_t render_mma_smem_bytes();
cudaError_t launch_render_mma(const CamArgs& cam, const UpliftWs& ws, int slot, const int32_t* topk_idx,
                              const float* topk_val, int K, int C, void* out, int out_bf16, float* out_T,
                              int32_t* out_last, cudaStream_t st);
cudaError_t launch_render_tiles(const CamArgs& cam, const UpliftWs& ws, int slot, const int32_t* topk_idx,
                                const float* topk_val, int K, int C, void* out, int out_bf16, float* out_T,
                                int32_t* out_last, cudaStream_t st);
size_t render_bwd_smem_bytes(int C, int K);
cudaError_t launch_render_bwd(const CamArgs& cam, const UpliftWs& ws, int slot, const int32_t* topk_idx,
                              const float* topk_val, int K, int C, const float* dL_dcodes, float* d_val,
                              float* d_opacity, cudaStream_t st);
constexpr int kOutBF16 = 0, kOutF32 = 1, kOutCos = 2, kOutRel = 3;
struct GemmEpi {
  int M, N, K;
  int mode;              // kOutBF16 / kOutF32 / kOutCos / kOutRel
  void* out;             // kOutRel: the relevancy [M, N - n_canon] (ldo = N - n_canon, a multiple of 4)
  int64_t ldo;           // elements
  float* rownorm2;       // kOutBF16: accumulated squared row norms (may be null); kOutCos, kOutRel: input
  const float* colnorm;  // kOutCos, kOutRel: column norms
  int n_canon = 0;       // kOutRel (N <= 32): the first n_canon columns are the canonical phrases
  float alpha = 0.0f;    // kOutRel: softmax temperature of Eq. 9
  int* status;
  int stall_loads = 0;   // self-test only: the producer issues no loads, so the bounded waits run out
  // Fused query (mode kOutBF16): every CTA takes whole row blocks and, after
  // a block's N columns, one more unit of sim_n (16 or 32) columns against
  // the operand Gt (bf16 [sim_n, K]); that unit's epilogue writes, with the
  // row's squared norm summed over the block's rounded features, the cosine
  // (sim_mode kOutCos, colnorm = the sim_n column norms) or the relevancy
  // (kOutRel, with n_canon and alpha) to sim_out [M, sim_ldo] (f32).
  int sim_n = 0;
  int sim_mode = 0;
  void* sim_out = nullptr;
  int64_t sim_ldo = 0;
  int store = 1;  // 0: the kOutBF16 rows are not written (their norms and the fused unit still are)
};
cudaError_t launch_gemm_bf16(const void* A, const void* Bt, const GemmEpi& ep, cudaStream_t st);
// launch_gemm_bf16 with the fused query unit (ep.sim_n > 0; Gt bf16 [sim_n, K]).
cudaError_t launch_gemm_bf16_query(const void* A, const void* Bt, const void* Gt, const GemmEpi& ep,
                                   cudaStream_t st);
// Gt[q][c] = bf16(sum_d text[q][d] codebook[c][d]) (FP32 sums) and tnorm[q] = |text_q| (FP32).
cudaError_t launch_text_codebook(const float* text, const float* codebook, int Q, int C, int D, void* Gt,
                                 float* tnorm, cudaStream_t st);
cudaError_t launch_f32_to_bf16(const float* x, void* y, int64_t n, cudaStream_t st);
cudaError_t launch_transpose_bf16(const float* B, void* Bt, int Cdim, int D, cudaStream_t st);
cudaError_t launch_row_norm_bf16(const void* X, int64_t R, int D, float* out, int squared, cudaStream_t st);
bool gemm_tma_available();
int gemm_timeout_selftest(void* workspace, size_t ws_bytes, cudaStream_t st);
cudaError_t launch_sgemm(const float* A, const float* B, bool b_transposed, float* out, int64_t M, int N, int K,
                         const float* rownorm2, const float* colnorm2, cudaStream_t st);
cudaError_t launch_row_norm2_f32(const float* X, int64_t R, int D, float* out, cudaStream_t st);
// ld: row stride of accum / comp in floats (C for a plain [n, C] accumulator).
cudaError_t launch_topk(const float* accum, const float* comp, int64_t n, int C, int K, int32_t* idx, float* val,
                        float* entropy, cudaStream_t st, int64_t ld = 0);
size_t entropy_filter_state_bytes();
int entropy_filter_run(const float* H, int64_t n, int64_t keep, int K, int32_t* idx, float* val, uint8_t* mask,
                       void* workspace, cudaStream_t st);
cudaError_t launch_region_targets(const int32_t* ci, const float* cv, int R, int s, const float* codebook, int C,
                                  int D, float* target, int* status, cudaStream_t st);
cudaError_t launch_l2_grad(const void* F, int F_bf16, int64_t P, int D, const int32_t* rmap, int R,
                           const float* target, void* dF, int dF_bf16, double* loss, int* status, cudaStream_t st);
cudaError_t launch_relevancy(const float* sim, int64_t P, int ncols, int n_canon, float alpha, float* R,
                             cudaStream_t st);
cudaError_t launch_code_topk(const int32_t* ci, const float* cv, int64_t R, int s, int K,
                             int32_t* ci_out, float* cv_out, cudaStream_t st);

}  // namespace scoup
