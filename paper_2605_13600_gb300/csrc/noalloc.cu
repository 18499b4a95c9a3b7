// noalloc.cu -- scoup_uplift_noalloc: the uplift with its scratch in a
// fixed, library-owned device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory: a host application whose
// memory manager owns every device allocation and hands out no scratch
// buffers, or a plugin that runs inside such a host and has no allocator to
// call.  They can still pass their inputs and outputs; the scratch this call
// needs lives in g_uplift_scratch below, a file-scope __device__ array that
// every GPU which loads this library holds until the process exits.
#include <cuda.h>
#include <stdio.h>

#include <mutex>

#include "scoup_internal.cuh"

namespace scoup {
namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_uplift_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// The driver's current context (through the runtime's entry-point query, so
// the library needs no link against the driver library); null if unknown.
CUcontext current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
    looked = true;
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of g_uplift_scratch on the current device (the host-side
// name of the array is not a device address).  It is looked up once per
// device and context: after a device reset the runtime loads the library's
// module again in a new context, the array gets a new address, and the
// cached one is replaced.
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_uplift_scratch);  // also creates the context if there is none yet
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = current_context();
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace scoup

extern "C" {

size_t scoup_uplift_noalloc_max_bytes(void) { return scoup::kNoAllocScratchBytes; }

int scoup_uplift_noalloc(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                         const int32_t* region_maps, const int64_t* map_offsets, int32_t R_total,
                         const int32_t* code_idx, const float* code_val, int32_t s, int32_t C,
                         int32_t K, float* accum, int32_t accum_mode, int32_t* topk_idx,
                         float* topk_val, scoup_stats* stats, void* stream) {
  if (!scene || scene->n < 0 || V < 0 || (V > 0 && !cams)) {
    // let scoup_uplift produce the precise message
    return scoup_uplift(scene, cams, V, region_maps, map_offsets, R_total, code_idx, code_val, s, C, K,
                        accum, accum_mode, topk_idx, topk_val, nullptr, 0, stats, stream);
  }
  int maxw = 1, maxh = 1;
  for (int v = 0; v < V; ++v) {
    if (cams[v].width > maxw) maxw = cams[v].width;
    if (cams[v].height > maxh) maxh = cams[v].height;
  }
  // one view pipeline: every byte after the fixed part goes to the tile lists
  const size_t fixed = scoup::uplift_required_bytes(scene->n, cams, V, s, K, R_total, 0);
  if (fixed > scoup::kNoAllocScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "scoup_uplift_noalloc: %lld Gaussians at %dx%d need %zu bytes of scratch before tile lists; "
             "the fixed array holds %zu", (long long)scene->n, maxw, maxh, fixed,
             scoup::kNoAllocScratchBytes);
    return scoup::set_error(SCOUP_ERR_INVALID_ARG, msg);
  }
  void* scratch = nullptr;
  cudaError_t e = scoup::scratch_address(&scratch);
  if (e != cudaSuccess)
    return scoup::set_error(SCOUP_ERR_CUDA, cudaGetErrorString(e));
  scoup_stats local;
  const scoup::UpliftCall c{scene, cams, V, region_maps, map_offsets, R_total, code_idx, code_val, s, C, K,
                            accum, accum_mode, topk_idx, topk_val};
  const scoup::WsHeader* hdr = nullptr;
  const int rc = scoup::uplift_call(c, scratch, scoup::kNoAllocScratchBytes, 8, &hdr, (cudaStream_t)stream, 1);
  if (rc != SCOUP_OK) return rc;
  return scoup::uplift_stats(hdr, stats ? stats : &local, (cudaStream_t)stream);
}

}  // extern "C"
