// api.cu -- C ABI entry points: validation, workspace carve-up, launch order.
#include <algorithm>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "drain.cuh"

namespace scoup {

std::atomic<long long> g_launches{0};

namespace {

// ---- optional per-phase CUDA-event timing -------------------------------
struct EventPair {
  int phase;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<EventPair> g_prof_pending;
std::vector<cudaEvent_t> g_prof_pool;
double g_prof_ms[SCOUP_NUM_PHASES];
long long g_prof_n[SCOUP_NUM_PHASES];

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one launch (or launch group) of a phase with events on `st`.
struct PhaseScope {
  int phase;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  PhaseScope(int ph, cudaStream_t s) : phase(ph), st(s) {
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    a = prof_event();
    cudaEventRecord(a, st);
  }
  ~PhaseScope() {
    if (!a) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t b = prof_event();
    cudaEventRecord(b, st);
    g_prof_pending.push_back({phase, a, b});
  }
};

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(SCOUP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int tiles_of(int w, int h) { return ((w + kTile - 1) / kTile) * ((h + kTile - 1) / kTile); }

// Workspace = shared part (header, Morton-ordered scene copy, codes) + one
// per-view part for each view pipeline (records, depth, rectangles, tile
// counters) + the key lists, split evenly between the pipelines.
size_t shared_bytes(int64_t n, int64_t code_rows_k) {
  const size_t un = (size_t)n;
  size_t b = align_up(sizeof(WsHeader));
  b += 2 * align_up(sizeof(float) * 3 * un);              // spatially ordered means, scales
  b += align_up(sizeof(float) * 4 * un);                  // quats
  b += 4 * align_up(sizeof(float) * un);                  // opacity, tau, orig, cell
  b += align_up(reorder_scratch_bytes());
  b += 2 * align_up((size_t)code_rows_k * 4);             // filtered codes (s > K)
  return b;
}

size_t lane_bytes(int64_t n, int max_tiles) {
  const size_t un = (size_t)n;
  size_t b = align_up(sizeof(ProjRec) * un);              // proj
  b += align_up(sizeof(uint32_t) * un);                   // depth
  b += align_up(sizeof(ushort4) * un);                    // rect
  b += 4 * align_up(sizeof(uint32_t) * ((size_t)max_tiles + 1));
  b += align_up(binning_run_base_bytes(n));               // binning: reserved-run offsets
  b += align_up(sizeof(float) * kTilePixels * (size_t)max_tiles);  // per-pixel state between slabs
  b += align_up((size_t)max_tiles);                       // tile done flags
  b += align_up(sizeof(uint32_t) * kDepthBuckets);        // depth histogram
  return b;
}

// Fixed part of the uplift workspace (everything but the key lists) for `lanes` view pipelines.
size_t uplift_fixed_bytes(int64_t n, int max_tiles, int64_t code_rows_k, int lanes = 1) {
  return shared_bytes(n, code_rows_k) + (size_t)lanes * lane_bytes(n, max_tiles);
}

}  // namespace

size_t carve_scene_part(void* base, int64_t n, int64_t code_rows_k, UpliftWs* w, int32_t** codes_i,
                        float** codes_v) {
  char* p = (char*)base;
  size_t off = 0;
  const size_t un = (size_t)n;
  auto take = [&](size_t sz) { char* q = p + off; off += align_up(sz); return (void*)q; };
  w->hdr = (WsHeader*)take(sizeof(WsHeader));
  w->sp.means = (float*)take(sizeof(float) * 3 * un);
  w->sp.scales = (float*)take(sizeof(float) * 3 * un);
  w->sp.quats = (float*)take(sizeof(float) * 4 * un);
  w->sp.opacity = (float*)take(sizeof(float) * un);
  w->sp.tau = (float*)take(sizeof(float) * un);
  w->sp.orig = (int32_t*)take(sizeof(int32_t) * un);
  w->cell = (uint32_t*)take(sizeof(uint32_t) * un);
  w->cells_scratch = (uint32_t*)take(reorder_scratch_bytes());
  *codes_i = (int32_t*)take((size_t)code_rows_k * 4);
  *codes_v = (float*)take((size_t)code_rows_k * 4);
  return off;
}

size_t carve_view_part(void* base, int64_t n, int max_tiles, UpliftWs* w) {
  char* p = (char*)base;
  size_t off = 0;
  const size_t un = (size_t)n;
  auto take = [&](size_t sz) { char* q = p + off; off += align_up(sz); return (void*)q; };
  w->max_tiles = max_tiles;
  w->proj = (ProjRec*)take(sizeof(ProjRec) * un);
  w->depth = (uint32_t*)take(sizeof(uint32_t) * un);
  w->rect = (ushort4*)take(sizeof(ushort4) * un);
  w->tile_count = (uint32_t*)take(sizeof(uint32_t) * ((size_t)max_tiles + 1));
  w->tile_glob = (uint32_t*)take(sizeof(uint32_t) * ((size_t)max_tiles + 1));
  w->run_base = (uint32_t*)take(binning_run_base_bytes(n));
  w->tile_start = (uint32_t*)take(sizeof(uint32_t) * ((size_t)max_tiles + 1));
  w->tile_fill = (uint32_t*)take(sizeof(uint32_t) * ((size_t)max_tiles + 1));
  w->pix_state = (float*)take(sizeof(float) * kTilePixels * (size_t)max_tiles);
  w->tile_done = (uint8_t*)take((size_t)max_tiles);
  w->dhist = (uint32_t*)take(sizeof(uint32_t) * kDepthBuckets);
  return off;
}

namespace {

// Carves `lanes` view pipelines out of the workspace; out[l] share the header
// and the scene copy.
void carve_lanes(void* ws, size_t bytes, int64_t n, int max_tiles, int64_t code_rows_k, int lanes,
                 int32_t** codes_i, float** codes_v, UpliftWs* out) {
  UpliftWs w;
  char* p = (char*)ws;
  size_t off = carve_scene_part(p, n, code_rows_k, &w, codes_i, codes_v);
  for (int l = 0; l < lanes; ++l) {
    out[l] = w;
    off += carve_view_part(p + off, n, max_tiles, &out[l]);
  }
  const int64_t keys_each = bytes > off ? (int64_t)((bytes - off) / sizeof(unsigned long long) / lanes) : 0;
  for (int l = 0; l < lanes; ++l) {
    out[l].keys = (unsigned long long*)(p + off) + (size_t)l * (size_t)keys_each;
    out[l].dup_capacity = keys_each;
  }
}

UpliftWs carve(void* ws, size_t bytes, int64_t n, int max_tiles, int64_t code_rows_k,
               int32_t** codes_i, float** codes_v) {
  UpliftWs w;
  carve_lanes(ws, bytes, n, max_tiles, code_rows_k, 1, codes_i, codes_v, &w);
  return w;
}

}  // namespace

int num_sms() {
  static std::atomic<int> cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

namespace {

// The library's second stream for the odd views of an uplift (one per host
// thread and device, created on first use).
cudaStream_t view_lane_stream() {
  thread_local cudaStream_t streams[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev] = nullptr;
  return streams[dev];
}

// The library's stream for staging host region maps (one per device and host thread).
cudaStream_t map_copy_stream() {
  thread_local cudaStream_t streams[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev] = nullptr;
  return streams[dev];
}

// The library's streams of the chunked form beyond the caller's and the view
// lane stream: [0] the second chunk lane, [1], [2] the lanes' second
// projection streams (one set per host thread and device).
cudaStream_t chunk_stream(int i) {
  thread_local cudaStream_t streams[64][3] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || i < 0 || i >= 3) return nullptr;
  if (!streams[dev][i] && cudaStreamCreateWithFlags(&streams[dev][i], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev][i] = nullptr;
  return streams[dev][i];
}

// Chunked form of one scene: kChunkLanes lanes of kChunkViews views per
// chunk, i.e. kChunkLanes x kChunkViews view parts in the workspace.
constexpr int kChunkLanes = 2, kChunkViews = 8;

// Bytes of the chunked layout with `dup` keys per view part.
size_t chunked_bytes(int64_t n, int max_tiles, int64_t code_rows_k, int64_t dup) {
  const size_t part = align_up(sizeof(WsHeader)) + lane_bytes(n, max_tiles) +
                      align_up(sizeof(unsigned long long) * (size_t)dup);
  return shared_bytes(n, code_rows_k) + (size_t)(kChunkLanes * kChunkViews) * part +
         align_up(sizeof(unsigned) * kChunkLanes);
}

// Depth slabs of the uplift.  Splitting a view into front-to-back slabs bins
// far fewer (Gaussian, tile) pairs (3 slabs at the 5% and 20% depth quantiles
// list 13% of the pairs of a 1M-Gaussian 988x731 view), but every slab pays a
// fixed cost of about 25 us per binning kernel plus a second per-tile setup,
// which measured more than the pairs it saves: one slab is the default.
SlabPlan uplift_slab_plan() {
  SlabPlan p;
  p.nslabs = 1;
  return p;
}

CamArgs cam_args(const scoup_camera& c) {
  CamArgs a;
  memcpy(a.vm, c.viewmat, sizeof(a.vm));
  a.fx = c.fx; a.fy = c.fy; a.cx = c.cx; a.cy = c.cy;
  a.width = c.width; a.height = c.height;
  a.gx = (c.width + kTile - 1) / kTile;
  a.gy = (c.height + kTile - 1) / kTile;
  return a;
}

int check_scene(const scoup_scene* sc) {
  if (!sc) return fail(SCOUP_ERR_INVALID_ARG, "scene is NULL");
  if (sc->n < 0 || sc->n > 0x7fffffffLL) return fail(SCOUP_ERR_INVALID_ARG, "scene n=%lld out of range", (long long)sc->n);
  if (sc->n > 0 && (!sc->means || !sc->scales || !sc->quats || !sc->opacity))
    return fail(SCOUP_ERR_INVALID_ARG, "scene arrays must be non-NULL when n > 0");
  if (sc->n > 0 && ((uintptr_t)sc->quats & 15u))
    return fail(SCOUP_ERR_INVALID_ARG, "scene quats must be 16-byte aligned");
  return SCOUP_OK;
}

int check_cams(const scoup_camera* cams, int V, int* max_tiles) {
  if (V < 0) return fail(SCOUP_ERR_INVALID_ARG, "V=%d < 0", V);
  if (V > 0 && !cams) return fail(SCOUP_ERR_INVALID_ARG, "cams is NULL");
  int mt = 1;
  for (int v = 0; v < V; ++v) {
    const scoup_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 65535 * kTile || c.height > 65535 * kTile)
      return fail(SCOUP_ERR_INVALID_ARG, "camera %d: bad size %dx%d", v, c.width, c.height);
    if (!(c.fx > 0.0f) || !(c.fy > 0.0f))
      return fail(SCOUP_ERR_INVALID_ARG, "camera %d: focal lengths must be > 0", v);
    const int t = tiles_of(c.width, c.height);
    if (t > mt) mt = t;
  }
  *max_tiles = mt;
  return SCOUP_OK;
}

void read_header(const WsHeader& h, scoup_stats* st) {
  st->visible = (int64_t)h.visible;
  st->duplicates = (int64_t)h.duplicates;
  st->evaluated_pairs = (int64_t)h.evaluated;
  st->contributions = (int64_t)h.contributions;
  st->flushes = (int64_t)h.flushes;
  st->atomics = (int64_t)h.atomics;
  st->listed = (int64_t)h.listed;
  st->max_dups_view = h.max_dups_view;
  st->split_windows = (int64_t)h.split_windows;
  st->status = SCOUP_OK;
  if (h.status & kStatCapacity) st->status = SCOUP_ERR_CAPACITY;
  else if (h.status & kStatDeviceCheck) st->status = SCOUP_ERR_DEVICE_CHECK;
  else if (h.status & kStatTimeout) st->status = SCOUP_ERR_TIMEOUT;
}

int finish_with_stats(const WsHeader* dev_hdr, scoup_stats* stats, cudaStream_t st) {
  WsHeader h;
  cudaError_t e = cudaMemcpyAsync(&h, dev_hdr, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "read stats");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  read_header(h, stats);
  if (stats->status == SCOUP_ERR_CAPACITY)
    return fail(SCOUP_ERR_CAPACITY, "tile-list capacity exceeded (largest view needs %d pairs)", h.max_dups_view);
  if (stats->status == SCOUP_ERR_DEVICE_CHECK)
    return fail(SCOUP_ERR_DEVICE_CHECK, "region or atom id out of range");
  if (stats->status == SCOUP_ERR_TIMEOUT)
    return fail(SCOUP_ERR_TIMEOUT, "a bounded device wait gave up");
  return SCOUP_OK;
}

}  // namespace
}  // namespace scoup

namespace scoup {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

// The views of one scene in chunks (SCOUP_UPLIFT_CHUNKED): view v goes to
// chunk v / kChunkViews on lane chunk % kChunkLanes; each chunk is projected
// and binned into the lane's view parts, composited by one drain launch and
// merged into the scene header sw.hdr.  The scene part (header, Morton-ordered
// copy) is set up; the view parts follow it in the workspace.  With host
// region maps (c.maps_on_host) view part q reads its map from ring slot q:
// a lane's copies for a chunk wait for the lane's previous drain (the last
// reader of its slots) and the chunk's drain waits for the copies; projection
// and binning do not read the maps and run meanwhile.
static int uplift_views_chunked(const UpliftCall& c, const int32_t* region_maps, int32_t R_total, const UpliftWs& sw,
                                void* workspace, size_t ws_bytes, int max_tiles, int64_t code_rows_k,
                                const int32_t* ci, const float* cv, int s_eff, float* comp, int warp_w,
                                cudaStream_t st) {
  const int64_t n = c.scene->n;
  const int V = c.V;
  constexpr int kParts = kChunkLanes * kChunkViews;
  // the layout: scene part, kParts x (header, view part, keys), lane counters
  const size_t fixed = chunked_bytes(n, max_tiles, code_rows_k, 0);
  if (ws_bytes < fixed + (size_t)kParts * 256)
    return fail(SCOUP_ERR_OOM, "workspace too small for the chunked form: %zu < %zu bytes before tile lists", ws_bytes,
                fixed + (size_t)kParts * 256);
  const size_t keys_each = (ws_bytes - fixed) / kParts / 256 * 256;
  char* p = (char*)workspace;
  size_t off = shared_bytes(n, code_rows_k);
  UpliftWs parts[kParts];
  DrainViewInit init[kParts];
  for (int q = 0; q < kParts; ++q) {
    UpliftWs& w = parts[q];
    w = sw;
    w.hdr = (WsHeader*)(p + off);
    off += align_up(sizeof(WsHeader));
    off += carve_view_part(p + off, n, max_tiles, &w);
    w.keys = (unsigned long long*)(p + off);
    w.dup_capacity = (int64_t)(keys_each / sizeof(unsigned long long));
    off += keys_each;
    init[q] = DrainViewInit{w.hdr, w.tile_count, w.tile_glob, w.dhist};
  }
  unsigned* counters = (unsigned*)(p + off);
  cudaError_t e;
  if ((e = launch_view_init(init, kParts, max_tiles, st)) != cudaSuccess) return cuda_fail(e, "view parts");
  // streams: lane 0 is `st`, lane 1 a library stream; each lane has a second projection stream
  const cudaStream_t lane_st[kChunkLanes] = {st, chunk_stream(0)};
  const cudaStream_t aux_st[kChunkLanes] = {chunk_stream(1), chunk_stream(2)};
  if (!lane_st[1] || !aux_st[0] || !aux_st[1]) return fail(SCOUP_ERR_CUDA, "could not create the chunk streams");
  cudaEvent_t ev[2 + 2 * kChunkLanes] = {};
  for (cudaEvent_t& x : ev)
    if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) {
      for (cudaEvent_t y : ev)
        if (y) cudaEventDestroy(y);
      return cuda_fail(e, "chunk events");
    }
  const cudaEvent_t fork = ev[0], join = ev[1];
  // host maps: copy stream forked from `st`; ready[l] = lane l's chunk maps are staged,
  // used[l] = lane l's last drain has been enqueued after them
  cudaStream_t cps = nullptr;
  cudaEvent_t mev[2 + 2 * kChunkLanes] = {};
  auto destroy_events = [&]() {
    for (cudaEvent_t y : ev) cudaEventDestroy(y);
    for (cudaEvent_t y : mev)
      if (y) cudaEventDestroy(y);
  };
  if (c.maps_on_host) {
    cps = map_copy_stream();
    bool ok = cps != nullptr;
    for (cudaEvent_t& x : mev) ok = ok && cudaEventCreateWithFlags(&x, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventRecord(mev[0], st) == cudaSuccess && cudaStreamWaitEvent(cps, mev[0], 0) == cudaSuccess;
    if (!ok) {
      destroy_events();
      return fail(SCOUP_ERR_CUDA, "map copy stream");
    }
  }
  int rc = SCOUP_OK;
  const int nchunks = (V + kChunkViews - 1) / kChunkViews;
  const bool lane1 = nchunks > 1;
  if (lane1 && ((e = cudaEventRecord(fork, st)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(lane_st[1], fork, 0)) != cudaSuccess))
    rc = cuda_fail(e, "chunk lanes");
  TileJob jobs[kChunkViews];
  uint32_t tile0[kChunkViews];
  UpliftWs views[kChunkViews];
  const scoup_scene* scenes[kChunkViews];
  for (int ch = 0; ch < nchunks && rc == SCOUP_OK; ++ch) {
    const int lane = ch % kChunkLanes;
    const int v0 = ch * kChunkViews, nv = std::min(kChunkViews, V - v0);
    uint32_t items = 0;
    for (int k = 0; k < nv; ++k) {
      const int v = v0 + k;
      const UpliftWs& w = parts[lane * kChunkViews + k];
      TileJob& J = jobs[k];
      J = TileJob();
      J.cam = cam_args(c.cams[v]);
      J.lc = LevelCodes();
      J.lc.L = 1;
      J.lc.s_tot = s_eff;
      J.lc.rmap[0] = c.maps_on_host ? c.map_stage + (size_t)(lane * kChunkViews + k) * c.map_stage_cap
                                    : region_maps + c.map_offsets[v];
      J.lc.ci[0] = ci;
      J.lc.cv[0] = cv;
      J.lc.s[0] = s_eff;
      J.lc.R[0] = R_total;
      J.proj = w.proj;
      J.keys = w.keys;
      J.tile_start = w.tile_start;
      J.accum = c.accum;
      J.comp = comp;
      J.hdr = w.hdr;
      J.scene_hdr = sw.hdr;
      J.slot = (ch / kChunkLanes) & 1;
      J.C = c.C;
      J.tiles = J.cam.gx * J.cam.gy;
      J.scene = 0;
      tile0[k] = items;
      items += (uint32_t)J.tiles;
      views[k] = w;
      scenes[k] = c.scene;
    }
    ChunkStreams cs{lane_st[lane], aux_st[lane], ev[2 + 2 * lane], ev[3 + 2 * lane]};
    if (c.maps_on_host) {
      // stage the chunk's maps into the lane's slots once the lane's previous drain has run
      cudaEvent_t ready = mev[2 + 2 * lane], used = mev[3 + 2 * lane];
      if (ch >= kChunkLanes && (e = cudaStreamWaitEvent(cps, used, 0)) != cudaSuccess) rc = cuda_fail(e, "map copy");
      for (int k = 0; k < nv && rc == SCOUP_OK; ++k) {
        const int v = v0 + k;
        const size_t bytes = sizeof(int32_t) * (size_t)c.cams[v].width * (size_t)c.cams[v].height;
        if ((e = cudaMemcpyAsync((void*)jobs[k].lc.rmap[0], region_maps + c.map_offsets[v], bytes,
                                 cudaMemcpyHostToDevice, cps)) != cudaSuccess)
          rc = cuda_fail(e, "region map copy");
      }
      if (rc == SCOUP_OK && (e = cudaEventRecord(ready, cps)) != cudaSuccess) rc = cuda_fail(e, "map copy");
      if (rc != SCOUP_OK) break;
      cs.before_drain = ready;
      cs.after_drain = used;
    }
    rc = run_chunk(jobs, tile0, nv, views, scenes, counters + lane, comp != nullptr, warp_w, cs);
  }
  if (c.maps_on_host &&
      ((e = cudaEventRecord(mev[1], cps)) != cudaSuccess || (e = cudaStreamWaitEvent(st, mev[1], 0)) != cudaSuccess) &&
      rc == SCOUP_OK)
    rc = cuda_fail(e, "map copy stream");
  // join even on an error, so that a capture in progress stays well formed
  if (lane1 && ((e = cudaEventRecord(join, lane_st[1])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess) && rc == SCOUP_OK)
    rc = cuda_fail(e, "chunk lanes");
  destroy_events();
  return rc;
}

int uplift_call(const UpliftCall& c, void* workspace, size_t ws_bytes, int warp_w, const WsHeader** hdr_out,
                cudaStream_t st, int view_lanes) {
  const scoup_scene* scene = c.scene;
  const scoup_camera* cams = c.cams;
  const int32_t V = c.V, C = c.C, K = c.K, accum_mode = c.accum_mode;
  const int64_t* map_offsets = c.map_offsets;
  // the semantic levels (one for the single-level form)
  scoup_level lv[kMaxLevels];
  int L = 1;
  if (c.L <= 0) {
    lv[0] = scoup_level{c.region_maps, c.R_total, c.code_idx, c.code_val, c.s};
  } else {
    if (c.L > kMaxLevels || !c.levels) return fail(SCOUP_ERR_INVALID_ARG, "L=%d outside [1, %d]", c.L, kMaxLevels);
    L = c.L;
    for (int l = 0; l < L; ++l) lv[l] = c.levels[l];
  }
  const int32_t R_total = lv[0].R_total, s = lv[0].s;
  const int32_t* region_maps = lv[0].region_maps;
  const int32_t* code_idx = lv[0].code_idx;
  const float* code_val = lv[0].code_val;
  float* accum = c.accum;
  int32_t* topk_idx = c.topk_idx;
  float* topk_val = c.topk_val;
  int rc = check_scene(scene);
  if (rc) return rc;
  int max_tiles = 1;
  if ((rc = check_cams(cams, V, &max_tiles))) return rc;
  if (C < 1 || C > 1024) return fail(SCOUP_ERR_INVALID_ARG, "C=%d outside [1, 1024]", C);
  if (K < 1 || K > C) return fail(SCOUP_ERR_INVALID_ARG, "K=%d outside [1, C=%d]", K, C);
  int s_tot = 0;
  for (int l = 0; l < L; ++l) {
    if (lv[l].s < 1 || lv[l].s > 1024) return fail(SCOUP_ERR_INVALID_ARG, "s=%d outside [1, 1024]", lv[l].s);
    if (lv[l].R_total < 0) return fail(SCOUP_ERR_INVALID_ARG, "R_total=%d < 0", lv[l].R_total);
    if (V > 0 && !lv[l].region_maps) return fail(SCOUP_ERR_INVALID_ARG, "region maps of level %d are NULL", l);
    if (V > 0 && lv[l].R_total > 0 && (!lv[l].code_idx || !lv[l].code_val))
      return fail(SCOUP_ERR_INVALID_ARG, "code table of level %d is NULL", l);
    if (L > 1 && lv[l].s > K)
      return fail(SCOUP_ERR_INVALID_ARG, "level %d: s=%d > K=%d (levels take codes of at most K entries)", l,
                  lv[l].s, K);
    if (L > 1 && lv[l].R_total >= (1 << 21) - 1)
      return fail(SCOUP_ERR_INVALID_ARG, "level %d: R_total=%d above 2^21 - 2", l, lv[l].R_total);
    s_tot += lv[l].s;
  }
  if (L > 1 && s_tot > 64) return fail(SCOUP_ERR_INVALID_ARG, "levels: sum of s = %d above 64", s_tot);
  const int Crow = L * C;
  if (accum_mode & ~(SCOUP_ACCUM_CONTINUE | SCOUP_ACCUM_COMPENSATED | SCOUP_UPLIFT_CHUNKED))
    return fail(SCOUP_ERR_INVALID_ARG,
                "accum_mode=%d: only SCOUP_ACCUM_CONTINUE, SCOUP_ACCUM_COMPENSATED and SCOUP_UPLIFT_CHUNKED", accum_mode);
  const bool chunked = (accum_mode & SCOUP_UPLIFT_CHUNKED) != 0;
  if (chunked && c.L > 0)
    return fail(SCOUP_ERR_INVALID_ARG, "SCOUP_UPLIFT_CHUNKED is a mode of the single-level uplift calls");
  if (scene->n > 0 && !accum) return fail(SCOUP_ERR_INVALID_ARG, "accum is NULL");
  if ((topk_idx == nullptr) != (topk_val == nullptr))
    return fail(SCOUP_ERR_INVALID_ARG, "topk_idx and topk_val must both be given or both be NULL");
  if (V > 0 && (!region_maps || !map_offsets)) return fail(SCOUP_ERR_INVALID_ARG, "region maps are NULL");
  for (int v = 0; v < V; ++v)
    if (map_offsets[v] < 0) return fail(SCOUP_ERR_INVALID_ARG, "map_offsets[%d] < 0", v);
  if (!workspace) return fail(SCOUP_ERR_INVALID_ARG, "workspace is NULL");
  if (c.maps_on_host) {
    if (L != 1) return fail(SCOUP_ERR_INVALID_ARG, "host region maps take a single level");
    if (!c.map_stage) return fail(SCOUP_ERR_INVALID_ARG, "no staging ring for host region maps");
    for (int v = 0; v < V; ++v)
      if ((int64_t)cams[v].width * cams[v].height > c.map_stage_cap)
        return fail(SCOUP_ERR_INVALID_ARG, "view %d is larger than the staging ring's slots", v);
  }
  const int64_t code_rows_k = (L == 1 && s > K) ? (int64_t)R_total * K : 0;
  const size_t fixed = uplift_fixed_bytes(scene->n, max_tiles, code_rows_k);
  if (ws_bytes < fixed)
    return fail(SCOUP_ERR_OOM, "workspace too small: %zu < %zu bytes before tile lists", ws_bytes, fixed);
  if (chunked && ws_bytes < chunked_bytes(scene->n, max_tiles, code_rows_k, 0) + (size_t)kChunkLanes * kChunkViews * 256)
    return fail(SCOUP_ERR_OOM, "workspace too small for the chunked form: %zu < %zu bytes before tile lists", ws_bytes,
                chunked_bytes(scene->n, max_tiles, code_rows_k, 0) + (size_t)kChunkLanes * kChunkViews * 256);

  // two view pipelines (even / odd views on two streams) when the workspace holds them
  const int lanes =
      (!chunked && view_lanes >= 2 && V >= 2 && ws_bytes >= uplift_fixed_bytes(scene->n, max_tiles, code_rows_k, 2) + 64) ? 2 : 1;
  int32_t* fci = nullptr;
  float* fcv = nullptr;
  UpliftWs wsl[2];
  carve_lanes(workspace, ws_bytes, scene->n, max_tiles, code_rows_k, lanes, &fci, &fcv, wsl);
  const UpliftWs& ws = wsl[0];
  const int64_t n = scene->n;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  const bool compensated = (accum_mode & SCOUP_ACCUM_COMPENSATED) != 0;
  float* comp = compensated ? accum + (size_t)n * (size_t)Crow : nullptr;
  if (n > 0 && !(accum_mode & SCOUP_ACCUM_CONTINUE) &&
      (e = cudaMemsetAsync(accum, 0, sizeof(float) * (size_t)n * (size_t)Crow * (compensated ? 2 : 1), st)) !=
          cudaSuccess)
    return cuda_fail(e, "memset accum");
  for (int l = 0; l < (chunked ? 0 : lanes); ++l)
    if ((e = cudaMemsetAsync(wsl[l].tile_glob, 0, sizeof(uint32_t) * ((size_t)max_tiles + 1), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(wsl[l].tile_count, 0, sizeof(uint32_t) * ((size_t)max_tiles + 1), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(wsl[l].dhist, 0, sizeof(uint32_t) * kDepthBuckets, st)) != cudaSuccess)
      return cuda_fail(e, "memset");
  const SlabPlan plan = uplift_slab_plan();
  const int32_t* ci = code_idx;
  const float* cv = code_val;
  int s_eff = s;
  if (L == 1 && s > K && R_total > 0) {
    PhaseScope ps(SCOUP_PHASE_CODE_TOPK, st);
    if ((e = launch_code_topk(code_idx, code_val, R_total, s, K, fci, fcv, st)) != cudaSuccess)
      return cuda_fail(e, "code top-k");
    ci = fci;
    cv = fcv;
    s_eff = K;
  }
  if (n > 0 && V > 0 && chunked) {
    {
      PhaseScope ps(SCOUP_PHASE_TAU, st);
      if ((e = launch_reorder(*scene, ws, st)) != cudaSuccess) return cuda_fail(e, "reorder");
    }
    const int rcc = uplift_views_chunked(c, region_maps, R_total, ws, workspace, ws_bytes, max_tiles, code_rows_k, ci,
                                         cv, s_eff, comp, warp_w, st);
    if (rcc != SCOUP_OK) return rcc;
  }
  if (n > 0 && V > 0 && !chunked) {
    {
      PhaseScope ps(SCOUP_PHASE_TAU, st);
      if ((e = launch_reorder(*scene, ws, st)) != cudaSuccess) return cuda_fail(e, "reorder");
    }
    // view v runs in pipeline v % lanes; the second pipeline forks from and
    // joins back into `st` through events (graph capture follows them)
    cudaStream_t sts[2] = {st, st};
    cudaEvent_t fork = nullptr, join = nullptr;
    if (lanes == 2) {
      sts[1] = view_lane_stream();
      if (!sts[1]) return fail(SCOUP_ERR_CUDA, "could not create the second view stream");
      if ((e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventRecord(fork, st)) != cudaSuccess || (e = cudaStreamWaitEvent(sts[1], fork, 0)) != cudaSuccess) {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        return cuda_fail(e, "view streams");
      }
    }
    // host maps: copy stream forked from `st`; ready[q] = slot q holds its
    // view's map, used[q] = the tile kernel that read slot q has finished
    cudaStream_t cs = nullptr;
    cudaEvent_t cfork = nullptr, cjoin = nullptr, ready[kMapStageSlots] = {}, used[kMapStageSlots] = {};
    auto destroy_copy_events = [&]() {
      for (cudaEvent_t* ev : {&cfork, &cjoin}) if (*ev) cudaEventDestroy(*ev);
      for (int q = 0; q < kMapStageSlots; ++q) {
        if (ready[q]) cudaEventDestroy(ready[q]);
        if (used[q]) cudaEventDestroy(used[q]);
      }
    };
    if (c.maps_on_host) {
      cs = map_copy_stream();
      bool ok = cs != nullptr;
      ok = ok && cudaEventCreateWithFlags(&cfork, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&cjoin, cudaEventDisableTiming) == cudaSuccess;
      for (int q = 0; q < kMapStageSlots && ok; ++q)
        ok = cudaEventCreateWithFlags(&ready[q], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&used[q], cudaEventDisableTiming) == cudaSuccess;
      ok = ok && cudaEventRecord(cfork, st) == cudaSuccess && cudaStreamWaitEvent(cs, cfork, 0) == cudaSuccess;
      if (!ok) {
        destroy_copy_events();
        if (lanes == 2) { cudaEventDestroy(fork); cudaEventDestroy(join); }
        return fail(SCOUP_ERR_CUDA, "map copy stream");
      }
    }
    int rc_views = SCOUP_OK;
    for (int v = 0; v < V && rc_views == SCOUP_OK; ++v) {
      const int lane = v % lanes, slot = 2 * lane + ((v / lanes) & 1);
      const cudaStream_t vs = sts[lane];
      const UpliftWs& wv = wsl[lane];
      const CamArgs ca = cam_args(cams[v]);
      {
        PhaseScope ps(SCOUP_PHASE_PREPROCESS, vs);
        if ((e = launch_preprocess(*scene, ca, wv, slot, vs, &plan)) != cudaSuccess) { rc_views = cuda_fail(e, "preprocess"); break; }
      }
      const int q = v % kMapStageSlots;
      if (c.maps_on_host) {
        // the copy waits for the tile kernel that last read slot q (view v - kMapStageSlots)
        const size_t bytes = sizeof(int32_t) * (size_t)cams[v].width * (size_t)cams[v].height;
        if ((v >= kMapStageSlots && (e = cudaStreamWaitEvent(cs, used[q], 0)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(c.map_stage + (size_t)q * c.map_stage_cap, region_maps + map_offsets[v], bytes,
                                 cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
            (e = cudaEventRecord(ready[q], cs)) != cudaSuccess) {
          rc_views = cuda_fail(e, "region map copy");
          break;
        }
      }
      {
        LevelCodes lc;
        lc.L = L;
        lc.s_tot = L == 1 ? s_eff : s_tot;
        for (int l = 0; l < kMaxLevels; ++l) {
          const bool on = l < L;
          lc.rmap[l] = on ? (c.maps_on_host ? c.map_stage + (size_t)q * c.map_stage_cap
                                            : lv[l].region_maps + map_offsets[v])
                          : nullptr;
          lc.ci[l] = on ? (L == 1 ? ci : lv[l].code_idx) : nullptr;
          lc.cv[l] = on ? (L == 1 ? cv : lv[l].code_val) : nullptr;
          lc.s[l] = on ? (L == 1 ? s_eff : lv[l].s) : 0;
          lc.R[l] = on ? lv[l].R_total : 0;
        }
        // slabs front to back: bin slab s (into the tiles still open), then composite it
        for (int sl = 0; sl < plan.nslabs && rc_views == SCOUP_OK; ++sl) {
          {
            PhaseScope ps(SCOUP_PHASE_BINNING, vs);
            if ((e = launch_binning(ca, n, wv, slot, vs, plan.nslabs > 1 ? sl : -1, sl == plan.nslabs - 1)) !=
                cudaSuccess)
              rc_views = cuda_fail(e, "binning");
          }
          if (rc_views != SCOUP_OK) break;
          // the first tile pass is the first reader of a staged region map
          if (sl == 0 && c.maps_on_host && (e = cudaStreamWaitEvent(vs, ready[q], 0)) != cudaSuccess) {
            rc_views = cuda_fail(e, "region map copy");
            break;
          }
          PhaseScope ps(SCOUP_PHASE_UPLIFT_TILES, vs);
          if ((e = launch_uplift_tiles(ca, wv, slot, lc, C, Crow, accum, comp, warp_w, vs, sl, plan.nslabs)) !=
              cudaSuccess)
            rc_views = cuda_fail(e, "uplift tiles");
        }
        if (rc_views != SCOUP_OK) break;
      }
      if (c.maps_on_host && (e = cudaEventRecord(used[q], vs)) != cudaSuccess) {
        rc_views = cuda_fail(e, "region map copy");
        break;
      }
    }
    if (c.maps_on_host) {
      if ((e = cudaEventRecord(cjoin, cs)) != cudaSuccess || (e = cudaStreamWaitEvent(st, cjoin, 0)) != cudaSuccess)
        if (rc_views == SCOUP_OK) rc_views = cuda_fail(e, "map copy stream");
      destroy_copy_events();
    }
    if (lanes == 2) {
      // join even on an error, so that a capture in progress stays well formed
      if ((e = cudaEventRecord(join, sts[1])) != cudaSuccess || (e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess)
        if (rc_views == SCOUP_OK) rc_views = cuda_fail(e, "view streams");
      cudaEventDestroy(fork);
      cudaEventDestroy(join);
    }
    if (rc_views != SCOUP_OK) return rc_views;
  }
  if (topk_idx && n > 0) {
    PhaseScope ps(SCOUP_PHASE_TOPK, st);
    for (int l = 0; l < L; ++l)
      if ((e = launch_topk(accum + (size_t)l * C, comp ? comp + (size_t)l * C : nullptr, n, C, K,
                           topk_idx + (size_t)l * n * K, topk_val + (size_t)l * n * K, nullptr, st, Crow)) !=
          cudaSuccess)
        return cuda_fail(e, "top-k");
  }
  if (hdr_out) *hdr_out = ws.hdr;
  return SCOUP_OK;
}

size_t uplift_required_bytes(int64_t n, const scoup_camera* cams, int32_t V, int32_t s, int32_t K, int32_t R_total,
                             int64_t dup_capacity) {
  int max_tiles = 1;
  for (int v = 0; v < V; ++v) {
    const int t = tiles_of(cams[v].width, cams[v].height);
    if (t > max_tiles) max_tiles = t;
  }
  const int64_t code_rows_k = s > K ? (int64_t)R_total * K : 0;
  return uplift_fixed_bytes(n, max_tiles, code_rows_k) + sizeof(unsigned long long) * (size_t)dup_capacity;
}

int run_chunk(const TileJob* jobs, const uint32_t* tile0, int njobs, const UpliftWs* views,
              const scoup_scene* const* scenes, unsigned* counter, bool compensated, int warp_w,
              const ChunkStreams& cs) {
  auto fail_cuda = [](cudaError_t e, const char* where) { return cuda_fail(e, where); };
  if (njobs <= 0) return SCOUP_OK;
  if (njobs > kMaxDrainJobs) return set_error(SCOUP_ERR_INVALID_ARG, "more views in a chunk than one drain takes");
  cudaError_t e;
  int rc = SCOUP_OK;
  // the second stream starts after the lane's previous drain (the view parts are reused)
  const bool split = njobs > 1 && cs.as != nullptr;
  if (split && ((e = cudaEventRecord(cs.fork, cs.ls)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(cs.as, cs.fork, 0)) != cudaSuccess))
    return fail_cuda(e, "fork");
  for (int j = 0; j < njobs && rc == SCOUP_OK; ++j) {
    const cudaStream_t vs = (split && (j & 1)) ? cs.as : cs.ls;
    const TileJob& J = jobs[j];
    {
      PhaseScope ps(SCOUP_PHASE_PREPROCESS, vs);
      if ((e = launch_preprocess(*scenes[j], J.cam, views[j], J.slot, vs)) != cudaSuccess) {
        rc = fail_cuda(e, "preprocess");
        break;
      }
    }
    PhaseScope ps(SCOUP_PHASE_BINNING, vs);
    if ((e = launch_binning(J.cam, scenes[j]->n, views[j], J.slot, vs)) != cudaSuccess) rc = fail_cuda(e, "binning");
  }
  // join even on an error, so that a capture in progress stays well formed
  if (split && ((e = cudaEventRecord(cs.join, cs.as)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(cs.ls, cs.join, 0)) != cudaSuccess) && rc == SCOUP_OK)
    rc = fail_cuda(e, "join");
  if (rc != SCOUP_OK) return rc;
  if (cs.before_drain && (e = cudaStreamWaitEvent(cs.ls, cs.before_drain, 0)) != cudaSuccess)
    return fail_cuda(e, "region map copy");
  if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned), cs.ls)) != cudaSuccess) return fail_cuda(e, "counter");
  {
    PhaseScope ps(SCOUP_PHASE_UPLIFT_TILES, cs.ls);
    if ((e = launch_uplift_drain(jobs, tile0, njobs, counter, compensated, warp_w, cs.ls)) != cudaSuccess)
      return fail_cuda(e, "drain");
  }
  if ((e = launch_view_merge(jobs, njobs, cs.ls)) != cudaSuccess) return fail_cuda(e, "merge");
  if (cs.after_drain && (e = cudaEventRecord(cs.after_drain, cs.ls)) != cudaSuccess)
    return fail_cuda(e, "region map copy");
  return SCOUP_OK;
}

size_t uplift_scene_part_bytes(int64_t n, int64_t code_rows_k) { return shared_bytes(n, code_rows_k); }

size_t uplift_view_part_bytes(int64_t n, int max_tiles) { return lane_bytes(n, max_tiles); }

CamArgs camera_args(const scoup_camera& c) { return cam_args(c); }

int check_scene_views(const scoup_scene* scene, const scoup_camera* cams, int32_t V, int* max_tiles) {
  const int rc = check_scene(scene);
  return rc ? rc : check_cams(cams, V, max_tiles);
}

int uplift_stats(const WsHeader* dev_hdr, scoup_stats* stats, cudaStream_t st) {
  return finish_with_stats(dev_hdr, stats, st);
}

void header_stats(const WsHeader& h, scoup_stats* stats) { read_header(h, stats); }



}  // namespace scoup

using namespace scoup;

extern "C" {

const char* scoup_version(void) { return "scoup-gb300 0.1.0 (sm_103a)"; }

const char* scoup_last_error(void) { return g_err.c_str(); }

size_t scoup_uplift_chunked_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                           int64_t dup_capacity) {
  if (n < 0 || max_width <= 0 || max_height <= 0 || dup_capacity < 0) return 0;
  return chunked_bytes(n, tiles_of(max_width, max_height), 0, dup_capacity);
}

size_t scoup_uplift_host_maps_chunked_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                                     int64_t dup_capacity) {
  if (n < 0 || max_width <= 0 || max_height <= 0 || dup_capacity < 0) return 0;
  return align_up(sizeof(int32_t) * (size_t)(kChunkLanes * kChunkViews) * (size_t)max_width * (size_t)max_height) +
         chunked_bytes(n, tiles_of(max_width, max_height), 0, dup_capacity);
}

size_t scoup_uplift_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                   int64_t dup_capacity) {
  if (n < 0 || max_width <= 0 || max_height <= 0 || dup_capacity < 0) return 0;
  return uplift_fixed_bytes(n, tiles_of(max_width, max_height), 0, 2) +
         2 * sizeof(unsigned long long) * (size_t)dup_capacity;
}

int scoup_uplift_plan(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                      void* workspace, size_t ws_bytes, int64_t* max_dups, void* stream) {
  int rc = check_scene(scene);
  if (rc) return rc;
  int max_tiles = 1;
  if ((rc = check_cams(cams, V, &max_tiles))) return rc;
  if (!max_dups) return fail(SCOUP_ERR_INVALID_ARG, "max_dups is NULL");
  if (!workspace) return fail(SCOUP_ERR_INVALID_ARG, "workspace is NULL");
  if (ws_bytes < uplift_fixed_bytes(scene->n, max_tiles, 0))
    return fail(SCOUP_ERR_OOM, "workspace too small: %zu < %zu bytes", ws_bytes,
                uplift_fixed_bytes(scene->n, max_tiles, 0));
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* ci = nullptr;
  float* cv = nullptr;
  UpliftWs ws = carve(workspace, ws_bytes, scene->n, max_tiles, 0, &ci, &cv);
  cudaError_t e = cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = launch_reorder(*scene, ws, st)) != cudaSuccess) return cuda_fail(e, "reorder");
  int64_t best = 0;
  for (int v = 0; v < V; ++v) {
    const CamArgs ca = cam_args(cams[v]);
    if ((e = cudaMemsetAsync(&ws.hdr->duplicates, 0, sizeof(unsigned long long), st)) != cudaSuccess)
      return cuda_fail(e, "memset");
    if ((e = launch_preprocess(*scene, ca, ws, v & 1, st)) != cudaSuccess) return cuda_fail(e, "preprocess");
    unsigned long long d = 0;
    if ((e = cudaMemcpyAsync(&d, &ws.hdr->duplicates, sizeof(d), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "read");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "synchronize");
    if ((int64_t)d > best) best = (int64_t)d;
  }
  *max_dups = best;
  return SCOUP_OK;
}

int scoup_uplift(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                 const int32_t* region_maps, const int64_t* map_offsets, int32_t R_total,
                 const int32_t* code_idx, const float* code_val, int32_t s, int32_t C, int32_t K,
                 float* accum, int32_t accum_mode, int32_t* topk_idx, float* topk_val,
                 void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream) {
  const UpliftCall c{scene, cams, V, region_maps, map_offsets, R_total, code_idx, code_val, s, C, K,
                     accum, accum_mode, topk_idx, topk_val};
  const WsHeader* hdr = nullptr;
  const cudaStream_t st = (cudaStream_t)stream;
  const int rc = uplift_call(c, workspace, ws_bytes, 8, &hdr, st, 2);
  if (rc != SCOUP_OK) return rc;
  if (stats) return finish_with_stats(hdr, stats, st);
  return SCOUP_OK;
}

size_t scoup_uplift_host_maps_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                             int64_t dup_capacity) {
  const size_t up = scoup_uplift_workspace_size(n, max_width, max_height, dup_capacity);
  if (!up) return 0;
  return align_up(sizeof(int32_t) * kMapStageSlots * (size_t)max_width * (size_t)max_height) + up;
}

// Workspace: [staging ring of kMapStageSlots view maps][scoup_uplift workspace].
int scoup_uplift_host_maps(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                           const int32_t* host_region_maps, const int64_t* map_offsets, int32_t R_total,
                           const int32_t* code_idx, const float* code_val, int32_t s, int32_t C, int32_t K,
                           float* accum, int32_t accum_mode, int32_t* topk_idx, float* topk_val,
                           void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream) {
  if (V < 0) return fail(SCOUP_ERR_INVALID_ARG, "V=%d < 0", V);
  if (V > 0 && !cams) return fail(SCOUP_ERR_INVALID_ARG, "cams is NULL");
  if (!workspace) return fail(SCOUP_ERR_INVALID_ARG, "workspace is NULL");
  int64_t cap = 1;
  for (int v = 0; v < V; ++v) {
    if (cams[v].width <= 0 || cams[v].height <= 0)
      return fail(SCOUP_ERR_INVALID_ARG, "view %d: bad size %dx%d", v, cams[v].width, cams[v].height);
    cap = std::max(cap, (int64_t)cams[v].width * cams[v].height);
  }
  // one ring slot per view in flight: kMapStageSlots, or one per view part of the chunked form
  const int slots = (accum_mode & SCOUP_UPLIFT_CHUNKED) ? kChunkLanes * kChunkViews : kMapStageSlots;
  const size_t ring = align_up(sizeof(int32_t) * (size_t)slots * (size_t)cap);
  if (ws_bytes < ring) return fail(SCOUP_ERR_OOM, "workspace too small: %zu < %zu bytes of staging ring", ws_bytes, ring);
  UpliftCall c{scene, cams, V, host_region_maps, map_offsets, R_total, code_idx, code_val, s, C, K,
               accum, accum_mode, topk_idx, topk_val};
  c.maps_on_host = true;
  c.map_stage = (int32_t*)workspace;
  c.map_stage_cap = cap;
  const WsHeader* hdr = nullptr;
  const cudaStream_t st = (cudaStream_t)stream;
  const int rc = uplift_call(c, (char*)workspace + ring, ws_bytes - ring, 8, &hdr, st, 2);
  if (rc != SCOUP_OK) return rc;
  if (stats) return finish_with_stats(hdr, stats, st);
  return SCOUP_OK;
}

int scoup_uplift_levels(const scoup_scene* scene, const scoup_camera* cams, int32_t V, const int64_t* map_offsets,
                        const scoup_level* levels, int32_t L, int32_t C, int32_t K, float* accum,
                        int32_t accum_mode, int32_t* topk_idx, float* topk_val, void* workspace, size_t ws_bytes,
                        scoup_stats* stats, void* stream) {
  if (L < 1 || L > kMaxLevels || !levels) return fail(SCOUP_ERR_INVALID_ARG, "L=%d outside [1, %d]", L, kMaxLevels);
  UpliftCall c{scene, cams, V, levels[0].region_maps, map_offsets, levels[0].R_total, levels[0].code_idx,
               levels[0].code_val, levels[0].s, C, K, accum, accum_mode, topk_idx, topk_val};
  c.L = L;
  c.levels = levels;
  const WsHeader* hdr = nullptr;
  const cudaStream_t st = (cudaStream_t)stream;
  const int rc = uplift_call(c, workspace, ws_bytes, 8, &hdr, st, 2);
  if (rc != SCOUP_OK) return rc;
  if (stats) return finish_with_stats(hdr, stats, st);
  return SCOUP_OK;
}

int scoup_render(const scoup_scene* scene, const int32_t* topk_idx, const float* topk_val, int32_t K,
                 int32_t C, const scoup_camera* cam, void* out_codes, int32_t out_dtype, float* out_T,
                 int32_t* out_last, void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream) {
  int rc = check_scene(scene);
  if (rc) return rc;
  int max_tiles = 1;
  if ((rc = check_cams(cam, 1, &max_tiles))) return rc;
  if (C < 1 || C > 1024) return fail(SCOUP_ERR_INVALID_ARG, "C=%d outside [1, 1024]", C);
  if (K < 1 || K > C) return fail(SCOUP_ERR_INVALID_ARG, "K=%d outside [1, C=%d]", K, C);
  if (!out_codes) return fail(SCOUP_ERR_INVALID_ARG, "out_codes is NULL");
  if (out_dtype != 0 && out_dtype != 1) return fail(SCOUP_ERR_INVALID_ARG, "out_dtype must be 0 (f32) or 1 (bf16)");
  if (scene->n > 0 && (!topk_idx || !topk_val)) return fail(SCOUP_ERR_INVALID_ARG, "Top-K arrays are NULL");
  if (!workspace) return fail(SCOUP_ERR_INVALID_ARG, "workspace is NULL");
  if (render_smem_bytes(C, K) > 227 * 1024)
    return fail(SCOUP_ERR_INVALID_ARG, "C=%d needs more shared memory than a CTA has", C);
  const size_t fixed = uplift_fixed_bytes(scene->n, max_tiles, 0);
  if (ws_bytes < fixed)
    return fail(SCOUP_ERR_OOM, "workspace too small: %zu < %zu bytes before tile lists", ws_bytes, fixed);
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* fci = nullptr;
  float* fcv = nullptr;
  UpliftWs ws = carve(workspace, ws_bytes, scene->n, max_tiles, 0, &fci, &fcv);
  const int64_t n = scene->n;
  const CamArgs ca = cam_args(*cam);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = cudaMemsetAsync(ws.tile_glob, 0, sizeof(uint32_t) * ((size_t)max_tiles + 1), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(ws.tile_count, 0, sizeof(uint32_t) * ((size_t)max_tiles + 1), st)) != cudaSuccess)
    return cuda_fail(e, "memset");
  {
    PhaseScope ps(SCOUP_PHASE_TAU, st);
    if ((e = launch_reorder(*scene, ws, st)) != cudaSuccess) return cuda_fail(e, "reorder");
  }
  if (n > 0) {
    PhaseScope ps(SCOUP_PHASE_PREPROCESS, st);
    if ((e = launch_preprocess(*scene, ca, ws, 0, st)) != cudaSuccess) return cuda_fail(e, "preprocess");
  }
  {
    PhaseScope ps(SCOUP_PHASE_BINNING, st);
    if ((e = launch_binning(ca, n, ws, 0, st)) != cudaSuccess) return cuda_fail(e, "binning");
  }
  {
    PhaseScope ps(SCOUP_PHASE_RENDER, st);
    if ((e = launch_render_tiles(ca, ws, 0, topk_idx, topk_val, K, C, out_codes, out_dtype, out_T, out_last, st)) !=
        cudaSuccess)
      return cuda_fail(e, "render tiles");
  }
  if (stats) return finish_with_stats(ws.hdr, stats, st);
  return SCOUP_OK;
}

int scoup_render_backward(const scoup_scene* scene, const int32_t* topk_idx, const float* topk_val,
                          int32_t K, int32_t C, const scoup_camera* cam, const float* dL_dcodes,
                          float* d_topk_val, float* d_opacity, void* workspace, size_t ws_bytes,
                          scoup_stats* stats, void* stream) {
  int rc = check_scene(scene);
  if (rc) return rc;
  int max_tiles = 1;
  if ((rc = check_cams(cam, 1, &max_tiles))) return rc;
  if (C < 1 || C > 1024) return fail(SCOUP_ERR_INVALID_ARG, "C=%d outside [1, 1024]", C);
  if (K < 1 || K > C || K > 64) return fail(SCOUP_ERR_INVALID_ARG, "K=%d outside [1, min(C, 64)]", K);
  if (!dL_dcodes) return fail(SCOUP_ERR_INVALID_ARG, "dL_dcodes is NULL");
  if (scene->n > 0 && (!topk_idx || !topk_val || !d_topk_val || !d_opacity))
    return fail(SCOUP_ERR_INVALID_ARG, "Top-K or gradient arrays are NULL");
  if (!workspace) return fail(SCOUP_ERR_INVALID_ARG, "workspace is NULL");
  if (render_bwd_smem_bytes(C, K) > 227 * 1024)
    return fail(SCOUP_ERR_INVALID_ARG, "C=%d, K=%d need more shared memory than a CTA has", C, K);
  const size_t fixed = uplift_fixed_bytes(scene->n, max_tiles, 0);
  if (ws_bytes < fixed)
    return fail(SCOUP_ERR_OOM, "workspace too small: %zu < %zu bytes before tile lists", ws_bytes, fixed);
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* fci = nullptr;
  float* fcv = nullptr;
  UpliftWs ws = carve(workspace, ws_bytes, scene->n, max_tiles, 0, &fci, &fcv);
  const int64_t n = scene->n;
  const CamArgs ca = cam_args(*cam);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = cudaMemsetAsync(ws.tile_glob, 0, sizeof(uint32_t) * ((size_t)max_tiles + 1), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(ws.tile_count, 0, sizeof(uint32_t) * ((size_t)max_tiles + 1), st)) != cudaSuccess)
    return cuda_fail(e, "memset");
  {
    PhaseScope ps(SCOUP_PHASE_TAU, st);
    if ((e = launch_reorder(*scene, ws, st)) != cudaSuccess) return cuda_fail(e, "reorder");
  }
  if (n > 0) {
    PhaseScope ps(SCOUP_PHASE_PREPROCESS, st);
    if ((e = launch_preprocess(*scene, ca, ws, 0, st)) != cudaSuccess) return cuda_fail(e, "preprocess");
  }
  {
    PhaseScope ps(SCOUP_PHASE_BINNING, st);
    if ((e = launch_binning(ca, n, ws, 0, st)) != cudaSuccess) return cuda_fail(e, "binning");
  }
  {
    PhaseScope ps(SCOUP_PHASE_RENDER_BWD, st);
    if ((e = launch_render_bwd(ca, ws, 0, topk_idx, topk_val, K, C, dL_dcodes, d_topk_val, d_opacity, st)) !=
        cudaSuccess)
      return cuda_fail(e, "render backward");
  }
  if (stats) return finish_with_stats(ws.hdr, stats, st);
  return SCOUP_OK;
}

// ---- decode (Eq. 8) and similarity ---------------------------------------
static int64_t decode_chunk_rows(int64_t P) {
  const int64_t cap = 262144;
  const int64_t r = P < cap ? P : cap;
  return (r + 127) / 128 * 128;
}

size_t scoup_decode_workspace_size(int64_t P, int32_t C, int32_t D) {
  if (P < 0 || C <= 0 || D <= 0) return 0;
  return align_up(sizeof(WsHeader)) + align_up((size_t)D * C * 2) + align_up((size_t)decode_chunk_rows(P) * C * 2);
}

int scoup_decode(const void* codes, int32_t codes_dtype, int64_t P, int32_t C, const float* codebook, int32_t D,
                 void* features, int32_t out_dtype, float* feat_norm2, void* workspace, size_t ws_bytes,
                 void* stream) {
  if (P < 0 || P > 0x7fffffffLL) return fail(SCOUP_ERR_INVALID_ARG, "P=%lld outside [0, 2^31)", (long long)P);
  if (C < 8 || C % 8 || C > 4096) return fail(SCOUP_ERR_INVALID_ARG, "C=%d must be a multiple of 8 in [8, 4096]", C);
  if (D < 16 || D % 16) return fail(SCOUP_ERR_INVALID_ARG, "D=%d must be a positive multiple of 16", D);
  if (codes_dtype != 0 && codes_dtype != 1) return fail(SCOUP_ERR_INVALID_ARG, "codes_dtype must be 0 (f32) or 1 (bf16)");
  if (out_dtype != 0 && out_dtype != 1) return fail(SCOUP_ERR_INVALID_ARG, "out_dtype must be 0 (f32) or 1 (bf16)");
  if (P > 0 && (!codes || !codebook || !features)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  if (((uintptr_t)codes & 15u) || ((uintptr_t)features & 15u))
    return fail(SCOUP_ERR_INVALID_ARG, "codes and features must be 16-byte aligned");
  if (!workspace || ws_bytes < scoup_decode_workspace_size(P, C, D))
    return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", scoup_decode_workspace_size(P, C, D));
  if (!gemm_tma_available()) return fail(SCOUP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)workspace;
  WsHeader* hdr = (WsHeader*)w;
  void* Bt = w + align_up(sizeof(WsHeader));
  void* Abuf = (char*)Bt + align_up((size_t)D * C * 2);
  cudaError_t e;
  PhaseScope ps(SCOUP_PHASE_DECODE, st);
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if (P == 0) return SCOUP_OK;
  if (feat_norm2 && (e = cudaMemsetAsync(feat_norm2, 0, sizeof(float) * (size_t)P, st)) != cudaSuccess)
    return cuda_fail(e, "memset");
  if ((e = launch_transpose_bf16(codebook, Bt, C, D, st)) != cudaSuccess) return cuda_fail(e, "codebook");
  // bf16 codes feed the GEMM directly (one launch); f32 codes are rounded to
  // bf16 chunk by chunk in the workspace first
  const int64_t chunk = codes_dtype == 1 ? P : decode_chunk_rows(P);
  for (int64_t r0 = 0; r0 < P; r0 += chunk) {
    const int64_t rows = P - r0 < chunk ? P - r0 : chunk;
    const void* A;
    if (codes_dtype == 0) {
      if ((e = launch_f32_to_bf16((const float*)codes + r0 * C, Abuf, rows * C, st)) != cudaSuccess)
        return cuda_fail(e, "convert");
      A = Abuf;
    } else {
      A = (const char*)codes + (size_t)r0 * C * 2;
    }
    GemmEpi ep;
    ep.M = (int)rows;
    ep.N = D;
    ep.K = C;
    ep.mode = out_dtype == 1 ? kOutBF16 : kOutF32;
    ep.out = (char*)features + (size_t)r0 * D * (out_dtype == 1 ? 2 : 4);
    ep.ldo = D;
    ep.rownorm2 = (out_dtype == 1 && feat_norm2) ? feat_norm2 + r0 : nullptr;
    ep.colnorm = nullptr;
    ep.status = &hdr->status;
    if ((e = launch_gemm_bf16(A, Bt, ep, st)) != cudaSuccess) return cuda_fail(e, "decode gemm");
  }
  return SCOUP_OK;
}

size_t scoup_render_decode_workspace_size(int64_t n, int32_t width, int32_t height, int32_t C, int32_t D,
                                          int64_t dup_capacity) {
  if (n < 0 || width <= 0 || height <= 0 || C <= 0 || D <= 0 || dup_capacity < 0) return 0;
  const int64_t P = (int64_t)width * height;
  const size_t dec = scoup_decode_workspace_size(P, C, D);
  const size_t up = scoup_uplift_workspace_size(n, width, height, dup_capacity);
  if (!dec || !up) return 0;
  return align_up(dec) + align_up((size_t)P * C * 2) + up;
}

// Workspace: [decode workspace][bf16 rendered codes, P x C][render workspace (the rest)].
int scoup_render_decode_fused(const scoup_scene* scene, const int32_t* topk_idx, const float* topk_val, int32_t K,
                              int32_t C, const scoup_camera* cam, const float* codebook, int32_t D, void* features,
                              int32_t out_dtype, float* feat_norm2, float* out_T, int32_t* out_last, void* workspace,
                              size_t ws_bytes, scoup_stats* stats, void* stream) {
  if (!cam) return fail(SCOUP_ERR_INVALID_ARG, "cam is NULL");
  if (cam->width <= 0 || cam->height <= 0)
    return fail(SCOUP_ERR_INVALID_ARG, "camera size %dx%d", cam->width, cam->height);
  if (C < 8 || C % 8 || C > 1024) return fail(SCOUP_ERR_INVALID_ARG, "C=%d must be a multiple of 8 in [8, 1024]", C);
  if (D < 16 || D % 16) return fail(SCOUP_ERR_INVALID_ARG, "D=%d must be a positive multiple of 16", D);
  if (!workspace) return fail(SCOUP_ERR_INVALID_ARG, "workspace is NULL");
  const int64_t P = (int64_t)cam->width * cam->height;
  const size_t dec = align_up(scoup_decode_workspace_size(P, C, D));
  const size_t wb = align_up((size_t)P * C * 2);
  if (ws_bytes < dec + wb) return fail(SCOUP_ERR_OOM, "workspace too small: %zu < %zu bytes before the render's", ws_bytes, dec + wb);
  char* w = (char*)workspace;
  void* What = w + dec;
  char* rws = w + dec + wb;
  int rc = scoup_render(scene, topk_idx, topk_val, K, C, cam, What, 1, out_T, out_last, rws, ws_bytes - dec - wb,
                        nullptr, stream);
  if (rc) return rc;
  rc = scoup_decode(What, 1, P, C, codebook, D, features, out_dtype, feat_norm2, w, dec, stream);
  if (rc) return rc;
  if (stats) {
    scoup_stats ds;
    const int r_render = finish_with_stats((const WsHeader*)rws, stats, (cudaStream_t)stream);
    if (r_render) return r_render;
    const int r_decode = finish_with_stats((const WsHeader*)w, &ds, (cudaStream_t)stream);
    if (r_decode) {
      stats->status = ds.status;
      return r_decode;
    }
  }
  return SCOUP_OK;
}

size_t scoup_similarity_workspace_size(int64_t P, int32_t D, int32_t Q) {
  if (P < 0 || D <= 0 || Q <= 0) return 0;
  return align_up(sizeof(WsHeader)) + align_up((size_t)Q * D * 2) + align_up((size_t)Q * 4) + align_up((size_t)P * 4);
}

int scoup_similarity(const void* features, int64_t P, int32_t D, const float* feat_norm2, const float* text,
                     int32_t Q, float* out, void* workspace, size_t ws_bytes, void* stream) {
  if (P < 0 || P > 0x7fffffffLL) return fail(SCOUP_ERR_INVALID_ARG, "P=%lld outside [0, 2^31)", (long long)P);
  if (D < 8 || D % 8) return fail(SCOUP_ERR_INVALID_ARG, "D=%d must be a positive multiple of 8", D);
  if (Q < 16 || Q % 16 || Q > 256) return fail(SCOUP_ERR_INVALID_ARG, "Q=%d must be a multiple of 16 in [16, 256]", Q);
  if (P > 0 && (!features || !text || !out)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  if (((uintptr_t)features & 15u) || ((uintptr_t)out & 15u))
    return fail(SCOUP_ERR_INVALID_ARG, "features and out must be 16-byte aligned");
  if (!workspace || ws_bytes < scoup_similarity_workspace_size(P, D, Q))
    return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", scoup_similarity_workspace_size(P, D, Q));
  if (!gemm_tma_available()) return fail(SCOUP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)workspace;
  WsHeader* hdr = (WsHeader*)w;
  void* tb = w + align_up(sizeof(WsHeader));
  float* tnorm = (float*)((char*)tb + align_up((size_t)Q * D * 2));
  float* fnorm2 = (float*)((char*)tnorm + align_up((size_t)Q * 4));
  cudaError_t e;
  PhaseScope ps(SCOUP_PHASE_SIMILARITY, st);
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if (P == 0) return SCOUP_OK;
  if ((e = launch_f32_to_bf16(text, tb, (int64_t)Q * D, st)) != cudaSuccess) return cuda_fail(e, "text");
  if ((e = launch_row_norm_bf16(tb, Q, D, tnorm, 0, st)) != cudaSuccess) return cuda_fail(e, "text norms");
  const float* rn2 = feat_norm2;
  if (!rn2) {
    if ((e = launch_row_norm_bf16(features, P, D, fnorm2, 1, st)) != cudaSuccess) return cuda_fail(e, "norms");
    rn2 = fnorm2;
  }
  GemmEpi ep;
  ep.M = (int)P;
  ep.N = Q;
  ep.K = D;
  ep.mode = kOutCos;
  ep.out = out;
  ep.ldo = Q;
  ep.rownorm2 = const_cast<float*>(rn2);
  ep.colnorm = tnorm;
  ep.status = &hdr->status;
  if ((e = launch_gemm_bf16(features, tb, ep, st)) != cudaSuccess) return cuda_fail(e, "similarity gemm");
  return SCOUP_OK;
}

int scoup_similarity_relevancy(const void* features, int64_t P, int32_t D, const float* feat_norm2,
                               const float* text, int32_t Q, int32_t n_canon, float alpha, float* R,
                               void* workspace, size_t ws_bytes, void* stream) {
  if (P < 0 || P > 0x7fffffffLL) return fail(SCOUP_ERR_INVALID_ARG, "P=%lld outside [0, 2^31)", (long long)P);
  if (D < 8 || D % 8) return fail(SCOUP_ERR_INVALID_ARG, "D=%d must be a positive multiple of 8", D);
  if (Q != 16 && Q != 32) return fail(SCOUP_ERR_INVALID_ARG, "Q=%d: the fused form takes 16 or 32 text vectors", Q);
  if (n_canon < 1 || n_canon >= Q || (Q - n_canon) % 4)
    return fail(SCOUP_ERR_INVALID_ARG, "n_canon=%d: need 1 <= n_canon < Q and Q - n_canon a multiple of 4", n_canon);
  if (!(alpha > 0.0f) || alpha > 3.0e38f) return fail(SCOUP_ERR_INVALID_ARG, "alpha must be positive and finite");
  if (P > 0 && (!features || !text || !R)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  if (((uintptr_t)features & 15u) || ((uintptr_t)R & 15u))
    return fail(SCOUP_ERR_INVALID_ARG, "features and R must be 16-byte aligned");
  if (!workspace || ws_bytes < scoup_similarity_workspace_size(P, D, Q))
    return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", scoup_similarity_workspace_size(P, D, Q));
  if (!gemm_tma_available()) return fail(SCOUP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)workspace;
  WsHeader* hdr = (WsHeader*)w;
  void* tb = w + align_up(sizeof(WsHeader));
  float* tnorm = (float*)((char*)tb + align_up((size_t)Q * D * 2));
  float* fnorm2 = (float*)((char*)tnorm + align_up((size_t)Q * 4));
  cudaError_t e;
  PhaseScope ps(SCOUP_PHASE_SIMILARITY, st);
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if (P == 0) return SCOUP_OK;
  if ((e = launch_f32_to_bf16(text, tb, (int64_t)Q * D, st)) != cudaSuccess) return cuda_fail(e, "text");
  if ((e = launch_row_norm_bf16(tb, Q, D, tnorm, 0, st)) != cudaSuccess) return cuda_fail(e, "text norms");
  const float* rn2 = feat_norm2;
  if (!rn2) {
    if ((e = launch_row_norm_bf16(features, P, D, fnorm2, 1, st)) != cudaSuccess) return cuda_fail(e, "norms");
    rn2 = fnorm2;
  }
  GemmEpi ep;
  ep.M = (int)P;
  ep.N = Q;
  ep.K = D;
  ep.mode = kOutRel;
  ep.out = R;
  ep.ldo = Q - n_canon;
  ep.rownorm2 = const_cast<float*>(rn2);
  ep.colnorm = tnorm;
  ep.n_canon = n_canon;
  ep.alpha = alpha;
  ep.status = &hdr->status;
  if ((e = launch_gemm_bf16(features, tb, ep, st)) != cudaSuccess) return cuda_fail(e, "similarity gemm");
  return SCOUP_OK;
}

size_t scoup_decode_query_workspace_size(int64_t P, int32_t C, int32_t D, int32_t Q) {
  if (P < 0 || C <= 0 || D <= 0 || Q <= 0) return 0;
  return align_up(scoup_decode_workspace_size(P, C, D)) + align_up((size_t)Q * C * 2) + align_up((size_t)Q * 4);
}

// Workspace: [decode workspace: header, bf16 codebook^T, bf16 code chunk][bf16 Gt = (text C^T), Q x C][|t_q|].
int scoup_decode_query(const void* codes, int32_t codes_dtype, int64_t P, int32_t C, const float* codebook,
                       int32_t D, const float* text, int32_t Q, int32_t n_canon, float alpha, void* features,
                       float* feat_norm2, float* out, void* workspace, size_t ws_bytes, void* stream) {
  if (P < 0 || P > 0x7fffffffLL) return fail(SCOUP_ERR_INVALID_ARG, "P=%lld outside [0, 2^31)", (long long)P);
  if (C < 8 || C % 8 || C > 4096) return fail(SCOUP_ERR_INVALID_ARG, "C=%d must be a multiple of 8 in [8, 4096]", C);
  if (D < 16 || D % 16) return fail(SCOUP_ERR_INVALID_ARG, "D=%d must be a positive multiple of 16", D);
  if (codes_dtype != 0 && codes_dtype != 1) return fail(SCOUP_ERR_INVALID_ARG, "codes_dtype must be 0 (f32) or 1 (bf16)");
  if (Q != 16 && Q != 32) return fail(SCOUP_ERR_INVALID_ARG, "Q=%d: the fused query takes 16 or 32 text vectors", Q);
  if (n_canon < 0 || n_canon >= Q || (n_canon > 0 && (Q - n_canon) % 4))
    return fail(SCOUP_ERR_INVALID_ARG, "n_canon=%d: need 0 (similarity) or 1 <= n_canon < Q with Q - n_canon a multiple of 4", n_canon);
  if (n_canon > 0 && (!(alpha > 0.0f) || alpha > 3.0e38f))
    return fail(SCOUP_ERR_INVALID_ARG, "alpha must be positive and finite");
  if (P > 0 && (!codes || !codebook || !text || !out)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  if (((uintptr_t)codes & 15u) || ((uintptr_t)features & 15u) || ((uintptr_t)out & 15u))
    return fail(SCOUP_ERR_INVALID_ARG, "codes, features and out must be 16-byte aligned");
  const size_t need = scoup_decode_query_workspace_size(P, C, D, Q);
  if (!workspace || ws_bytes < need) return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", need);
  if (!gemm_tma_available()) return fail(SCOUP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)workspace;
  WsHeader* hdr = (WsHeader*)w;
  void* Bt = w + align_up(sizeof(WsHeader));
  void* Abuf = (char*)Bt + align_up((size_t)D * C * 2);
  void* Gt = w + align_up(scoup_decode_workspace_size(P, C, D));
  float* tnorm = (float*)((char*)Gt + align_up((size_t)Q * C * 2));
  cudaError_t e;
  PhaseScope ps(SCOUP_PHASE_DECODE, st);
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if (P == 0) return SCOUP_OK;
  if ((e = launch_transpose_bf16(codebook, Bt, C, D, st)) != cudaSuccess) return cuda_fail(e, "codebook");
  if ((e = launch_text_codebook(text, codebook, Q, C, D, Gt, tnorm, st)) != cudaSuccess)
    return cuda_fail(e, "text x codebook");
  const int64_t ldq = n_canon > 0 ? Q - n_canon : Q;
  const int64_t chunk = codes_dtype == 1 ? P : decode_chunk_rows(P);
  for (int64_t r0 = 0; r0 < P; r0 += chunk) {
    const int64_t rows = P - r0 < chunk ? P - r0 : chunk;
    const void* A;
    if (codes_dtype == 0) {
      if ((e = launch_f32_to_bf16((const float*)codes + r0 * C, Abuf, rows * C, st)) != cudaSuccess)
        return cuda_fail(e, "convert");
      A = Abuf;
    } else {
      A = (const char*)codes + (size_t)r0 * C * 2;
    }
    GemmEpi ep;
    ep.M = (int)rows;
    ep.N = D;
    ep.K = C;
    ep.mode = kOutBF16;
    ep.out = features ? (char*)features + (size_t)r0 * D * 2 : nullptr;
    ep.ldo = D;
    ep.store = features ? 1 : 0;
    ep.rownorm2 = feat_norm2 ? feat_norm2 + r0 : nullptr;
    ep.colnorm = tnorm;
    ep.n_canon = n_canon;
    ep.alpha = alpha;
    ep.sim_n = Q;
    ep.sim_mode = n_canon > 0 ? kOutRel : kOutCos;
    ep.sim_out = out + r0 * ldq;
    ep.sim_ldo = ldq;
    ep.status = &hdr->status;
    if ((e = launch_gemm_bf16_query(A, Bt, Gt, ep, st)) != cudaSuccess) return cuda_fail(e, "decode + query gemm");
  }
  return SCOUP_OK;
}

size_t scoup_decode_backward_workspace_size(int64_t P, int32_t C, int32_t D) {
  if (P < 0 || C <= 0 || D <= 0) return 0;
  return align_up(sizeof(WsHeader)) + align_up((size_t)C * D * 2) + align_up((size_t)decode_chunk_rows(P) * D * 2);
}

int scoup_decode_backward(const void* dF, int32_t dF_dtype, int64_t P, int32_t D, const float* codebook, int32_t C,
                          float* dcodes, void* workspace, size_t ws_bytes, void* stream) {
  if (P < 0 || P > 0x7fffffffLL) return fail(SCOUP_ERR_INVALID_ARG, "P=%lld outside [0, 2^31)", (long long)P);
  if (C < 16 || C % 16 || C > 4096) return fail(SCOUP_ERR_INVALID_ARG, "C=%d must be a multiple of 16 in [16, 4096]", C);
  if (D < 8 || D % 8) return fail(SCOUP_ERR_INVALID_ARG, "D=%d must be a positive multiple of 8", D);
  if (dF_dtype != 0 && dF_dtype != 1) return fail(SCOUP_ERR_INVALID_ARG, "dF_dtype must be 0 (f32) or 1 (bf16)");
  if (P > 0 && (!dF || !codebook || !dcodes)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  if (((uintptr_t)dF & 15u) || ((uintptr_t)dcodes & 15u))
    return fail(SCOUP_ERR_INVALID_ARG, "dF and dcodes must be 16-byte aligned");
  if (!workspace || ws_bytes < scoup_decode_backward_workspace_size(P, C, D))
    return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", scoup_decode_backward_workspace_size(P, C, D));
  if (!gemm_tma_available()) return fail(SCOUP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)workspace;
  WsHeader* hdr = (WsHeader*)w;
  void* Bt = w + align_up(sizeof(WsHeader));  // the codebook rows are the K-major operand as they are
  void* Abuf = (char*)Bt + align_up((size_t)C * D * 2);
  cudaError_t e;
  PhaseScope ps(SCOUP_PHASE_DECODE, st);
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if (P == 0) return SCOUP_OK;
  if ((e = launch_f32_to_bf16(codebook, Bt, (int64_t)C * D, st)) != cudaSuccess) return cuda_fail(e, "codebook");
  const int64_t chunk = dF_dtype == 1 ? P : decode_chunk_rows(P);
  for (int64_t r0 = 0; r0 < P; r0 += chunk) {
    const int64_t rows = P - r0 < chunk ? P - r0 : chunk;
    const void* A;
    if (dF_dtype == 0) {
      if ((e = launch_f32_to_bf16((const float*)dF + r0 * D, Abuf, rows * D, st)) != cudaSuccess)
        return cuda_fail(e, "convert");
      A = Abuf;
    } else {
      A = (const char*)dF + (size_t)r0 * D * 2;
    }
    GemmEpi ep;
    ep.M = (int)rows;
    ep.N = C;
    ep.K = D;
    ep.mode = kOutF32;
    ep.out = dcodes + (size_t)r0 * C;
    ep.ldo = C;
    ep.rownorm2 = nullptr;
    ep.colnorm = nullptr;
    ep.status = &hdr->status;
    if ((e = launch_gemm_bf16(A, Bt, ep, st)) != cudaSuccess) return cuda_fail(e, "decode backward gemm");
  }
  return SCOUP_OK;
}

int scoup_decode_backward_fp32(const float* dF, int64_t P, int32_t D, const float* codebook, int32_t C,
                               float* dcodes, void* stream) {
  if (P < 0 || C < 1 || D < 1) return fail(SCOUP_ERR_INVALID_ARG, "bad sizes P=%lld C=%d D=%d", (long long)P, C, D);
  if (P > 0 && (!dF || !codebook || !dcodes)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  PhaseScope ps(SCOUP_PHASE_DECODE, (cudaStream_t)stream);
  const cudaError_t e = launch_sgemm(dF, codebook, true, dcodes, P, C, D, nullptr, nullptr, (cudaStream_t)stream);
  return e == cudaSuccess ? SCOUP_OK : cuda_fail(e, "sgemm");
}

size_t scoup_region_l2_grad_workspace_size(int32_t R, int32_t D) {
  if (R < 0 || D <= 0) return 0;
  return align_up(sizeof(WsHeader)) + align_up((size_t)(R > 0 ? R : 1) * D * 4);
}

int scoup_region_l2_grad(const void* F, int32_t F_dtype, int64_t P, int32_t D, const int32_t* region_map,
                         const int32_t* code_idx, const float* code_val, int32_t R, int32_t s,
                         const float* codebook, int32_t C, void* dF, int32_t dF_dtype, double* loss,
                         void* workspace, size_t ws_bytes, void* stream) {
  if (P < 0 || D < 1 || R < 0 || s < 1 || C < 1) return fail(SCOUP_ERR_INVALID_ARG, "bad sizes");
  if ((F_dtype != 0 && F_dtype != 1) || (dF_dtype != 0 && dF_dtype != 1))
    return fail(SCOUP_ERR_INVALID_ARG, "F_dtype and dF_dtype must be 0 (f32) or 1 (bf16)");
  if (P > 0 && (!F || !region_map || !dF || !codebook)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  if (R > 0 && (!code_idx || !code_val)) return fail(SCOUP_ERR_INVALID_ARG, "code table is NULL");
  if (!workspace || ws_bytes < scoup_region_l2_grad_workspace_size(R, D))
    return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", scoup_region_l2_grad_workspace_size(R, D));
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)workspace;
  WsHeader* hdr = (WsHeader*)w;
  float* target = (float*)(w + align_up(sizeof(WsHeader)));
  cudaError_t e;
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if (P == 0) return SCOUP_OK;
  if ((e = launch_region_targets(code_idx, code_val, R, s, codebook, C, D, target, &hdr->status, st)) != cudaSuccess)
    return cuda_fail(e, "region targets");
  if ((e = launch_l2_grad(F, F_dtype, P, D, region_map, R, target, dF, dF_dtype, loss, &hdr->status, st)) !=
      cudaSuccess)
    return cuda_fail(e, "loss gradient");
  return SCOUP_OK;
}

int scoup_decode_fp32(const float* codes, int64_t P, int32_t C, const float* codebook, int32_t D,
                      float* features, void* stream) {
  if (P < 0 || C < 1 || D < 1) return fail(SCOUP_ERR_INVALID_ARG, "bad sizes P=%lld C=%d D=%d", (long long)P, C, D);
  if (P > 0 && (!codes || !codebook || !features)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  cudaStream_t st = (cudaStream_t)stream;
  PhaseScope ps(SCOUP_PHASE_DECODE, st);
  const cudaError_t e = launch_sgemm(codes, codebook, false, features, P, D, C, nullptr, nullptr, st);
  return e == cudaSuccess ? SCOUP_OK : cuda_fail(e, "fp32 decode");
}

int scoup_similarity_fp32(const float* features, int64_t P, int32_t D, const float* text, int32_t Q, float* out,
                          void* workspace, size_t ws_bytes, void* stream) {
  if (P < 0 || D < 1 || Q < 1) return fail(SCOUP_ERR_INVALID_ARG, "bad sizes P=%lld D=%d Q=%d", (long long)P, D, Q);
  if (P > 0 && (!features || !text || !out)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  const size_t need = align_up(sizeof(WsHeader)) + align_up((size_t)Q * 4) + align_up((size_t)P * 4);
  if (!workspace || ws_bytes < need) return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", need);
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)workspace;
  float* tn2 = (float*)(w + align_up(sizeof(WsHeader)));
  float* fn2 = (float*)((char*)tn2 + align_up((size_t)Q * 4));
  cudaError_t e;
  PhaseScope ps(SCOUP_PHASE_SIMILARITY, st);
  if ((e = cudaMemsetAsync(w, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if (P == 0) return SCOUP_OK;
  if ((e = launch_row_norm2_f32(text, Q, D, tn2, st)) != cudaSuccess) return cuda_fail(e, "text norms");
  if ((e = launch_row_norm2_f32(features, P, D, fn2, st)) != cudaSuccess) return cuda_fail(e, "norms");
  if ((e = launch_sgemm(features, text, true, out, P, Q, D, fn2, tn2, st)) != cudaSuccess)
    return cuda_fail(e, "fp32 similarity");
  return SCOUP_OK;
}

int scoup_topk(const float* accum, int64_t n, int32_t C, int32_t K, int32_t* topk_idx,
               float* topk_val, void* stream) {
  if (n < 0) return fail(SCOUP_ERR_INVALID_ARG, "n < 0");
  if (C < 1 || C > 1024) return fail(SCOUP_ERR_INVALID_ARG, "C=%d outside [1, 1024]", C);
  if (K < 1 || K > C) return fail(SCOUP_ERR_INVALID_ARG, "K=%d outside [1, C=%d]", K, C);
  if (n > 0 && (!accum || !topk_idx || !topk_val)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  PhaseScope ps(SCOUP_PHASE_TOPK, (cudaStream_t)stream);
  cudaError_t e = launch_topk(accum, nullptr, n, C, K, topk_idx, topk_val, nullptr, (cudaStream_t)stream);
  return e == cudaSuccess ? SCOUP_OK : cuda_fail(e, "top-k");
}

int scoup_topk_entropy(const float* accum, const float* comp, int64_t n, int32_t C, int32_t K, int32_t* topk_idx,
                       float* topk_val, float* entropy, void* stream) {
  if (n < 0) return fail(SCOUP_ERR_INVALID_ARG, "n < 0");
  if (C < 1 || C > 1024) return fail(SCOUP_ERR_INVALID_ARG, "C=%d outside [1, 1024]", C);
  if (K < 1 || K > C) return fail(SCOUP_ERR_INVALID_ARG, "K=%d outside [1, C=%d]", K, C);
  if (n > 0 && (!accum || !topk_idx || !topk_val || !entropy)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  PhaseScope ps(SCOUP_PHASE_TOPK, (cudaStream_t)stream);
  cudaError_t e = launch_topk(accum, comp, n, C, K, topk_idx, topk_val, entropy, (cudaStream_t)stream);
  return e == cudaSuccess ? SCOUP_OK : cuda_fail(e, "top-k + entropy");
}

size_t scoup_entropy_filter_workspace_size(void) {
  return entropy_filter_state_bytes() < 1024 ? 1024 : entropy_filter_state_bytes();
}

int scoup_entropy_filter(const float* entropy, int64_t n, int64_t keep, int32_t K, int32_t* topk_idx,
                         float* topk_val, uint8_t* keep_mask, void* workspace, size_t ws_bytes, void* stream) {
  if (n < 0 || n > 0x7fffffffLL) return fail(SCOUP_ERR_INVALID_ARG, "n=%lld outside [0, 2^31)", (long long)n);
  if (keep < 0) return fail(SCOUP_ERR_INVALID_ARG, "keep < 0");
  if ((topk_idx == nullptr) != (topk_val == nullptr))
    return fail(SCOUP_ERR_INVALID_ARG, "topk_idx and topk_val must both be given or both be NULL");
  if (topk_idx && K < 1) return fail(SCOUP_ERR_INVALID_ARG, "K < 1");
  if (n > 0 && !entropy) return fail(SCOUP_ERR_INVALID_ARG, "entropy is NULL");
  if (!workspace || ws_bytes < scoup_entropy_filter_workspace_size())
    return fail(SCOUP_ERR_OOM, "workspace too small: need %zu bytes", scoup_entropy_filter_workspace_size());
  if (n == 0) return SCOUP_OK;
  if ((uintptr_t)workspace & 15u) return fail(SCOUP_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  return entropy_filter_run(entropy, n, keep, K, topk_idx, topk_val, keep_mask, workspace, (cudaStream_t)stream);
}

int scoup_relevancy(const float* sim, int64_t P, int32_t ncols, int32_t n_canon, float alpha, float* R,
                    void* stream) {
  if (P < 0) return fail(SCOUP_ERR_INVALID_ARG, "P < 0");
  if (n_canon < 1 || ncols <= n_canon) return fail(SCOUP_ERR_INVALID_ARG, "need 1 <= n_canon < ncols");
  if (!(alpha > 0.0f) || alpha > 3.0e38f) return fail(SCOUP_ERR_INVALID_ARG, "alpha must be positive and finite");
  if (P > 0 && (!sim || !R)) return fail(SCOUP_ERR_INVALID_ARG, "NULL array");
  PhaseScope ps(SCOUP_PHASE_SIMILARITY, (cudaStream_t)stream);
  cudaError_t e = launch_relevancy(sim, P, ncols, n_canon, alpha, R, (cudaStream_t)stream);
  return e == cudaSuccess ? SCOUP_OK : cuda_fail(e, "relevancy");
}

int scoup_selftest_gemm_timeout(void* workspace, size_t ws_bytes, void* stream) {
  if (!gemm_tma_available()) return fail(SCOUP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const int rc = gemm_timeout_selftest(workspace, ws_bytes, (cudaStream_t)stream);
  if (rc == SCOUP_ERR_TIMEOUT) return fail(rc, "tensor-core pipeline wait ran out (self-test, expected)");
  if (rc != SCOUP_OK) return fail(rc, "self-test could not run (workspace must hold 49408 bytes, 256-byte aligned)");
  return fail(SCOUP_ERR_DEVICE_CHECK, "self-test: the stalled pipeline did not report a timeout");
}

int scoup_read_stats(const void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream) {
  if (!workspace || ws_bytes < sizeof(WsHeader)) return fail(SCOUP_ERR_INVALID_ARG, "bad workspace");
  if (!stats) return fail(SCOUP_ERR_INVALID_ARG, "stats is NULL");
  return finish_with_stats((const WsHeader*)workspace, stats, (cudaStream_t)stream);
}

int scoup_profile_enable(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = enable != 0;
  return SCOUP_OK;
}

int scoup_profile_read(double* ms, int64_t* launches, int32_t nphases) {
  if (nphases < 0 || (nphases > 0 && (!ms || !launches)))
    return fail(SCOUP_ERR_INVALID_ARG, "bad profile output arrays");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (const EventPair& p : g_prof_pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e != cudaSuccess) return cuda_fail(e, "profile event");
    float t = 0.0f;
    cudaEventElapsedTime(&t, p.a, p.b);
    g_prof_ms[p.phase] += t;
    g_prof_n[p.phase] += 1;
    g_prof_pool.push_back(p.a);
    g_prof_pool.push_back(p.b);
  }
  g_prof_pending.clear();
  for (int i = 0; i < nphases && i < SCOUP_NUM_PHASES; ++i) {
    ms[i] = g_prof_ms[i];
    launches[i] = g_prof_n[i];
    g_prof_ms[i] = 0.0;
    g_prof_n[i] = 0;
  }
  return SCOUP_OK;
}

int64_t scoup_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
