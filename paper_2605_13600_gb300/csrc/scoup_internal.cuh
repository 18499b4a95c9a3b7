// scoup_internal.cuh -- shared definitions of the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/scoup.h"

#include <atomic>

namespace scoup {

// Kernel launches issued by the library (every launcher adds its count).
extern std::atomic<long long> g_launches;

constexpr int kTile = 16;            // 16x16 pixel tiles define binning membership (3DGS)
constexpr int kTilePixels = kTile * kTile;

// Device status bits (workspace header).
constexpr int kStatCapacity = 1;
constexpr int kStatDeviceCheck = 2;

// Workspace header: status word + counters, 256 bytes.
struct WsHeader {
  int32_t status;
  int32_t max_dups_view;
  int32_t pad[2];
  unsigned long long visible;
  unsigned long long duplicates;
  unsigned long long evaluated;
  unsigned long long contributions;
  unsigned long long flushes;
  unsigned long long atomics;
  unsigned long long reserved[24];
};
static_assert(sizeof(WsHeader) == 256, "header size");

// Projected Gaussian of one view, 32 bytes:
//   a = (mx, my, qa, qb), b = (qc, opacity, tau, unused)
// power(dx, dy) = dx*(qa*dx + qb*dy) + (qc*dy)*dy and the Gaussian is
// accepted at a pixel iff tau <= power <= 0  (tau: smallest float with
// o*exp(tau) >= 1/255).
struct __align__(16) ProjRec {
  float4 a;
  float4 b;
};

struct CamArgs {
  float vm[12];
  float fx, fy, cx, cy;
  int width, height;
  int gx, gy;  // tile grid
};

// Workspace carve-up for one uplift call.
struct UpliftWs {
  WsHeader* hdr;
  float* tau;               // [n] alpha-threshold exponent per Gaussian
  ProjRec* proj;            // [n]
  uint32_t* depth;          // [n] float bits of camera depth
  ushort4* rect;            // [n] tile rect (x_lo, y_lo, x_hi, y_hi), empty if culled
  uint32_t* tile_count;     // [max_tiles + 1]
  uint32_t* tile_start;     // [max_tiles + 1]
  uint32_t* tile_fill;      // [max_tiles]
  unsigned long long* keys; // [dup_capacity] (depth bits << 32 | gid)
  int64_t dup_capacity;
  int max_tiles;
};

// Launchers (each defined in its own translation unit).
cudaError_t launch_tau(const float* opacity, int64_t n, float* tau, cudaStream_t st);
cudaError_t launch_preprocess(const scoup_scene& sc, const CamArgs& cam, const UpliftWs& ws,
                              cudaStream_t st);
cudaError_t launch_binning(const CamArgs& cam, int64_t n, const UpliftWs& ws, cudaStream_t st);
cudaError_t launch_uplift_tiles(const CamArgs& cam, const UpliftWs& ws, const int32_t* rmap,
                                int32_t R_total, const int32_t* code_idx, const float* code_val,
                                int s, int C, float* accum, cudaStream_t st);
cudaError_t launch_topk(const float* accum, int64_t n, int C, int K, int32_t* idx, float* val,
                        cudaStream_t st);
cudaError_t launch_code_topk(const int32_t* ci, const float* cv, int64_t R, int s, int K,
                             int32_t* ci_out, float* cv_out, cudaStream_t st);

}  // namespace scoup
