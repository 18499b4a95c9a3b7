// batch.cu -- batched uplift of many scenes, each with its own views
// (Sec. 4.2, Eq. 5 and Eq. 6 per scene; the batching itself has no
// counterpart in the paper).
//
// A plan owns everything the batch needs on the device.  Scenes are spread
// over `lanes` CUDA streams, each with its own uplift workspace, by longest
// processing time first (estimated cost: views x largest per-view tile-pair
// count); inside a lane the scenes run one after another.  Small scenes and
// small views leave most SMs idle when run alone, so lanes overlap their
// preprocess, binning and tile kernels.  The first scoup_uplift_batched
// captures the whole batch (fork to the lanes, every launch of every scene,
// a device-side copy of each scene's counters, join) into one CUDA graph and
// later calls replay it with a single graph launch.
//
// The autotuner times every (lanes, tile-kernel warp block) pair on an evenly
// spaced sample of each scene's views and keeps the fastest; membership is
// always decided on the 16x16 tile, so the choice changes speed and the order
// of FP32 sums only.
#include <stdio.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "drain.cuh"

struct scoup_plan {
  std::vector<scoup_batch_item> items;
  int32_t C = 0, K = 0, accum_mode = 0;
  int device = 0;
  int lanes = 1;
  int warp_w = 8;
  int chunk = 0;                  // 0: scenes on lanes; > 0: chunks of this many views (drain.cu)
  bool tuned = false;
  std::vector<int64_t> max_dups;  // per scene
  std::vector<double> cost;       // per scene
  size_t lane_bytes = 0;          // bytes of one lane workspace
  std::vector<void*> lane_ws;
  std::vector<cudaStream_t> lane_st;
  std::vector<cudaEvent_t> join_ev;
  cudaEvent_t fork_ev = nullptr;
  cudaStream_t cap_st = nullptr;  // origin stream of the graph capture
  scoup::WsHeader* stats_dev = nullptr;  // [B]
  cudaGraphExec_t exec = nullptr;
  long long graph_kernels = 0;
  std::vector<scoup_tune_entry> tune;
  scoup::DrainLayout drain;       // device memory and schedule of the chunked form
};

namespace scoup {
namespace {

constexpr int kMaxLanes = 8;

int err(int code, const char* msg) { return set_error(code, msg); }

int cuda_err(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return set_error(SCOUP_ERR_CUDA, buf);
}

void drop_graph(scoup_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
  p->graph_kernels = 0;
}

// Lane workspaces, streams and events for `lanes` lanes (grows or shrinks).
int ensure_lanes(scoup_plan* p, int lanes) {
  cudaError_t e;
  while ((int)p->lane_ws.size() < lanes) {
    void* w = nullptr;
    if ((e = cudaMalloc(&w, p->lane_bytes)) != cudaSuccess) return cuda_err(e, "lane workspace");
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) {
      cudaFree(w);
      return cuda_err(e, "lane stream");
    }
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
      cudaFree(w);
      cudaStreamDestroy(s);
      return cuda_err(e, "lane event");
    }
    p->lane_ws.push_back(w);
    p->lane_st.push_back(s);
    p->join_ev.push_back(ev);
  }
  while ((int)p->lane_ws.size() > lanes) {
    cudaStreamSynchronize(p->lane_st.back());
    cudaFree(p->lane_ws.back());
    cudaStreamDestroy(p->lane_st.back());
    cudaEventDestroy(p->join_ev.back());
    p->lane_ws.pop_back();
    p->lane_st.pop_back();
    p->join_ev.pop_back();
  }
  return SCOUP_OK;
}

// Scenes of each lane, longest processing time first.
std::vector<std::vector<int>> assign(const scoup_plan* p, int lanes) {
  const int B = (int)p->items.size();
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p->cost[a] > p->cost[b]; });
  std::vector<std::vector<int>> out(lanes);
  std::vector<double> load(lanes, 0.0);
  for (int b : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    out[l].push_back(b);
    load[l] += p->cost[b];
  }
  return out;
}

// A view subset of one item: every step-th view (host copies of the cameras
// and offsets live in `cams` / `offs`).
struct ItemView {
  std::vector<scoup_camera> cams;
  std::vector<int64_t> offs;
};

ItemView sample_views(const scoup_batch_item& it, int max_views) {
  ItemView s;
  if (it.V <= 0) return s;
  const int take = max_views > 0 && max_views < it.V ? max_views : it.V;
  for (int k = 0; k < take; ++k) {
    const int v = (int)((int64_t)k * it.V / take);
    s.cams.push_back(it.cams[v]);
    s.offs.push_back(it.map_offsets[v]);
  }
  return s;
}

// Enqueue the batch (or a view sample of it) on the lanes, forked from and
// joined back into `st`.  copy_stats: append a device copy of each scene's
// counters to stats_dev.
int enqueue_batch(scoup_plan* p, int lanes, int warp_w, int sample, bool copy_stats, cudaStream_t st,
                  int chunk = 0) {
  cudaError_t e;
  if (chunk > 0) {
    const DrainLayout& d = p->drain;
    if (!d.mem || d.chunk != chunk || d.lanes != lanes || d.sample != sample)
      return err(SCOUP_ERR_INVALID_ARG, "chunked batch: layout not prepared for this configuration");
    return drain_enqueue(&p->drain, p->items, p->C, p->K, p->accum_mode, warp_w, p->lane_st.data(), p->join_ev.data(),
                         p->fork_ev, copy_stats ? p->stats_dev : nullptr, st);
  }
  if ((e = cudaEventRecord(p->fork_ev, st)) != cudaSuccess) return cuda_err(e, "fork");
  const auto groups = assign(p, lanes);
  std::vector<ItemView> views(p->items.size());
  for (int l = 0; l < lanes; ++l) {
    cudaStream_t ls = p->lane_st[l];
    if ((e = cudaStreamWaitEvent(ls, p->fork_ev, 0)) != cudaSuccess) return cuda_err(e, "fork wait");
    for (int b : groups[l]) {
      const scoup_batch_item& it = p->items[b];
      const scoup_camera* cams = it.cams;
      const int64_t* offs = it.map_offsets;
      int V = it.V;
      if (sample > 0) {
        views[b] = sample_views(it, sample);
        cams = views[b].cams.data();
        offs = views[b].offs.data();
        V = (int)views[b].cams.size();
      }
      const UpliftCall c{&it.scene, cams, V, it.region_maps, offs, it.R_total, it.code_idx, it.code_val, it.s,
                         p->C, p->K, it.accum, p->accum_mode, it.topk_idx, it.topk_val};
      const WsHeader* hdr = nullptr;
      const int rc = uplift_call(c, p->lane_ws[l], p->lane_bytes, warp_w, &hdr, ls);
      if (rc != SCOUP_OK) return rc;
      if (copy_stats &&
          (e = cudaMemcpyAsync(p->stats_dev + b, hdr, sizeof(WsHeader), cudaMemcpyDeviceToDevice, ls)) !=
              cudaSuccess)
        return cuda_err(e, "stats copy");
    }
    if ((e = cudaEventRecord(p->join_ev[l], ls)) != cudaSuccess) return cuda_err(e, "join");
    if ((e = cudaStreamWaitEvent(st, p->join_ev[l], 0)) != cudaSuccess) return cuda_err(e, "join wait");
  }
  return SCOUP_OK;
}

// Lays out the chunked form for (chunk, lanes, sample) unless it already is;
// synchronises the device, so never while capturing.
int ensure_drain(scoup_plan* p, int chunk, int lanes, int sample) {
  const DrainLayout& d = p->drain;
  if (d.mem && d.chunk == chunk && d.lanes == lanes && d.sample == sample) return SCOUP_OK;
  return drain_prepare(&p->drain, p->items, p->max_dups, p->C, p->K, p->accum_mode, chunk, lanes, sample);
}

// Captures the batch on the plan's own origin stream (the caller's stream may
// be the legacy default stream, which cannot be captured).
int capture(scoup_plan* p) {
  drop_graph(p);
  const cudaStream_t st = p->cap_st;
  cudaError_t e;
  if (p->chunk > 0) {
    const int rc = ensure_drain(p, p->chunk, p->lanes, 0);
    if (rc != SCOUP_OK) return rc;
  }
  if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_err(e, "begin capture");
  const long long l0 = g_launches.load();
  const int rc = enqueue_batch(p, p->lanes, p->warp_w, 0, true, st, p->chunk);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  const long long nk = g_launches.load() - l0;
  g_launches -= nk;  // counted again at every replay
  if (rc != SCOUP_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_err(e, "end capture");
  e = cudaGraphInstantiate(&p->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    p->exec = nullptr;
    return cuda_err(e, "graph instantiate");
  }
  p->graph_kernels = nk;
  return SCOUP_OK;
}

}  // namespace
}  // namespace scoup

using namespace scoup;

extern "C" {

int scoup_plan_create(const scoup_batch_item* items, int32_t B, int32_t C, int32_t K, int32_t accum_mode,
                      scoup_plan** plan_out, void* stream) {
  if (!plan_out) return err(SCOUP_ERR_INVALID_ARG, "plan_out is NULL");
  *plan_out = nullptr;
  if (B < 0 || (B > 0 && !items)) return err(SCOUP_ERR_INVALID_ARG, "bad batch (B < 0 or items NULL)");
  if (C < 1 || C > 1024 || K < 1 || K > C) return err(SCOUP_ERR_INVALID_ARG, "C or K out of range");
  if (accum_mode & ~(SCOUP_ACCUM_CONTINUE | SCOUP_ACCUM_COMPENSATED))
    return err(SCOUP_ERR_INVALID_ARG, "accum_mode: only SCOUP_ACCUM_CONTINUE and SCOUP_ACCUM_COMPENSATED");
  cudaStream_t st = (cudaStream_t)stream;
  scoup_plan* p = new scoup_plan();
  p->items.assign(items, items + B);
  p->C = C;
  p->K = K;
  p->accum_mode = accum_mode;
  cudaGetDevice(&p->device);
  cudaError_t e;
  int rc = SCOUP_OK;
  // exact per-view tile-pair counts of every scene (one planning workspace)
  size_t plan_bytes = 0;
  for (const scoup_batch_item& it : p->items) {
    if (it.V < 0 || (it.V > 0 && (!it.cams || !it.map_offsets))) {
      delete p;
      return err(SCOUP_ERR_INVALID_ARG, "batch item: bad views");
    }
    plan_bytes = std::max(plan_bytes, uplift_required_bytes(it.scene.n, it.cams, it.V, 1, 1, 0, 0));
  }
  void* tmp = nullptr;
  if (B > 0 && (e = cudaMalloc(&tmp, plan_bytes)) != cudaSuccess) {
    delete p;
    return cuda_err(e, "planning workspace");
  }
  for (int b = 0; b < B && rc == SCOUP_OK; ++b) {
    const scoup_batch_item& it = p->items[b];
    int64_t md = 0;
    rc = scoup_uplift_plan(&it.scene, it.cams, it.V, tmp, plan_bytes, &md, stream);
    p->max_dups.push_back(md);
    p->cost.push_back((double)it.V * (double)(md + it.scene.n));
  }
  if (tmp) cudaFree(tmp);
  if (rc != SCOUP_OK) {
    delete p;
    return rc;
  }
  for (int b = 0; b < B; ++b) {
    const scoup_batch_item& it = p->items[b];
    p->lane_bytes = std::max(p->lane_bytes, uplift_required_bytes(it.scene.n, it.cams, it.V, it.s, K, it.R_total,
                                                                  p->max_dups[b] + 1));
  }
  if ((e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&p->cap_st, cudaStreamNonBlocking)) != cudaSuccess ||
      (B > 0 && (e = cudaMalloc(&p->stats_dev, sizeof(WsHeader) * (size_t)B)) != cudaSuccess)) {
    scoup_plan_destroy(p);
    return cuda_err(e, "plan events / stats");
  }
  if (B > 0 && (e = cudaMemsetAsync(p->stats_dev, 0, sizeof(WsHeader) * (size_t)B, st)) != cudaSuccess) {
    scoup_plan_destroy(p);
    return cuda_err(e, "memset");
  }
  p->lanes = std::max(1, std::min(4, B));
  if ((rc = ensure_lanes(p, p->lanes)) != SCOUP_OK) {
    scoup_plan_destroy(p);
    return rc;
  }
  *plan_out = p;
  return SCOUP_OK;
}

int scoup_plan_set(scoup_plan* p, int32_t lanes, int32_t warp_w) {
  if (!p) return err(SCOUP_ERR_INVALID_ARG, "plan is NULL");
  if (lanes < 1 || lanes > kMaxLanes) return err(SCOUP_ERR_INVALID_ARG, "lanes outside [1, 8]");
  if (warp_w != 4 && warp_w != 8 && warp_w != 16) return err(SCOUP_ERR_INVALID_ARG, "warp_w must be 4, 8 or 16");
  drop_graph(p);
  const int rc = ensure_lanes(p, lanes);
  if (rc != SCOUP_OK) return rc;
  p->lanes = lanes;
  p->warp_w = warp_w;
  return SCOUP_OK;
}

int scoup_autotune(scoup_plan* p, int32_t sample_views, void* stream) {
  if (!p) return err(SCOUP_ERR_INVALID_ARG, "plan is NULL");
  if (p->accum_mode & SCOUP_ACCUM_CONTINUE)
    return err(SCOUP_ERR_INVALID_ARG, "autotune overwrites accum: not with SCOUP_ACCUM_CONTINUE");
  if (sample_views < 1) return err(SCOUP_ERR_INVALID_ARG, "sample_views < 1");
  cudaStream_t st = (cudaStream_t)stream;
  const int B = (int)p->items.size();
  if (B == 0) return SCOUP_OK;
  drop_graph(p);
  cudaError_t e;
  int rc = ensure_lanes(p, std::min(kMaxLanes, B));
  if (rc != SCOUP_OK) return rc;
  cudaEvent_t t0, t1;
  if ((e = cudaEventCreate(&t0)) != cudaSuccess) return cuda_err(e, "event");
  if ((e = cudaEventCreate(&t1)) != cudaSuccess) {
    cudaEventDestroy(t0);
    return cuda_err(e, "event");
  }
  p->tune.clear();
  double best = 1e300;
  int best_l = p->lanes, best_w = p->warp_w, best_c = 0;
  // one configuration: one warm-up, then the best of two timed runs
  auto try_config = [&](int lanes, int w, int chunk) {
    if (chunk > 0 && (rc = ensure_drain(p, chunk, lanes, sample_views)) != SCOUP_OK) return;
    float ms_best = 1e30f;
    for (int rep = 0; rep < 3 && rc == SCOUP_OK; ++rep) {
      if ((e = cudaEventRecord(t0, st)) != cudaSuccess) { rc = cuda_err(e, "event"); break; }
      rc = enqueue_batch(p, lanes, w, sample_views, true, st, chunk);
      if (rc != SCOUP_OK) break;
      if ((e = cudaEventRecord(t1, st)) != cudaSuccess || (e = cudaEventSynchronize(t1)) != cudaSuccess) {
        rc = cuda_err(e, "autotune timing");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (rep > 0) ms_best = std::min(ms_best, ms);
    }
    if (rc != SCOUP_OK) return;
    scoup_tune_entry te;
    te.lanes = lanes;
    te.warp_w = w;
    te.ms = ms_best;
    te.chunk_views = chunk;
    p->tune.push_back(te);
    if (ms_best < best) {
      best = ms_best;
      best_l = lanes;
      best_w = w;
      best_c = chunk;
    }
  };
  // scenes on lanes, every warp block; then the chunked form with the best warp block
  const int lane_opts[] = {1, 2, 4, 8};
  const int w_opts[] = {8, 16, 4};
  for (int lanes : lane_opts) {
    if (lanes > B) break;
    for (int w : w_opts)
      if (rc == SCOUP_OK) try_config(lanes, w, 0);
  }
  const int w_lane = best_w;
  const int chunk_opts[] = {4, 8, 16};
  for (int chunk : chunk_opts)
    for (int lanes : {1, 2, 4})
      if (rc == SCOUP_OK && lanes <= (int)p->lane_st.size()) try_config(lanes, w_lane, chunk);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc != SCOUP_OK) return rc;
  // the sample runs left every scene's counters in stats_dev: none may have failed
  std::vector<WsHeader> h(B);
  if ((e = cudaMemcpy(h.data(), p->stats_dev, sizeof(WsHeader) * (size_t)B, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_err(e, "read status");
  for (int b = 0; b < B; ++b)
    if (h[b].status) return err(SCOUP_ERR_DEVICE_CHECK, "a scene reported a device error while tuning");
  p->tuned = true;
  rc = scoup_plan_set(p, best_l, best_w);
  if (rc != SCOUP_OK) return rc;
  return scoup_plan_set_chunk(p, best_c);
}

int scoup_plan_set_chunk(scoup_plan* p, int32_t chunk_views) {
  if (!p) return err(SCOUP_ERR_INVALID_ARG, "plan is NULL");
  if (chunk_views < 0 || chunk_views > SCOUP_MAX_CHUNK_VIEWS)
    return err(SCOUP_ERR_INVALID_ARG, "chunk_views outside [0, 64]");
  if (chunk_views != p->chunk) drop_graph(p);
  p->chunk = chunk_views;
  return SCOUP_OK;
}

int scoup_uplift_batched(scoup_plan* p, int32_t flags, void* stream) {
  if (!p) return err(SCOUP_ERR_INVALID_ARG, "plan is NULL");
  if (flags & ~SCOUP_BATCH_EAGER) return err(SCOUP_ERR_INVALID_ARG, "unknown flags");
  cudaStream_t st = (cudaStream_t)stream;
  if (p->items.empty()) return SCOUP_OK;
  if (flags & SCOUP_BATCH_EAGER) {
    if (p->chunk > 0) {
      const int rc = ensure_drain(p, p->chunk, p->lanes, 0);
      if (rc != SCOUP_OK) return rc;
    }
    return enqueue_batch(p, p->lanes, p->warp_w, 0, true, st, p->chunk);
  }
  if (!p->exec) {
    const int rc = capture(p);
    if (rc != SCOUP_OK) return rc;
  }
  const cudaError_t e = cudaGraphLaunch(p->exec, st);
  if (e != cudaSuccess) return cuda_err(e, "graph launch");
  g_launches += p->graph_kernels;
  return SCOUP_OK;
}

int scoup_plan_stats(scoup_plan* p, scoup_stats* stats, void* stream) {
  if (!p || (!stats && !p->items.empty())) return err(SCOUP_ERR_INVALID_ARG, "plan or stats is NULL");
  const int B = (int)p->items.size();
  if (B == 0) return SCOUP_OK;
  std::vector<WsHeader> h(B);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h.data(), p->stats_dev, sizeof(WsHeader) * (size_t)B, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e, "read stats");
  int rc = SCOUP_OK;
  for (int b = 0; b < B; ++b) {
    header_stats(h[b], &stats[b]);
    if (stats[b].status != SCOUP_OK && rc == SCOUP_OK) rc = stats[b].status;
  }
  if (rc != SCOUP_OK) return err(rc, "a scene of the batch reported a device error (see its stats)");
  return SCOUP_OK;
}

int scoup_plan_info_get(const scoup_plan* p, scoup_plan_info* info) {
  if (!p || !info) return err(SCOUP_ERR_INVALID_ARG, "plan or info is NULL");
  info->lanes = p->lanes;
  info->warp_w = p->warp_w;
  info->tuned = p->tuned ? 1 : 0;
  info->graph_kernels = (int32_t)p->graph_kernels;
  info->workspace_bytes = (int64_t)(p->lane_bytes * p->lane_ws.size() + p->drain.bytes);
  info->chunk_views = p->chunk;
  info->n_tune = (int32_t)std::min<size_t>(p->tune.size(), SCOUP_MAX_TUNE);
  for (int i = 0; i < info->n_tune; ++i) info->tune[i] = p->tune[i];
  return SCOUP_OK;
}

int scoup_plan_destroy(scoup_plan* p) {
  if (!p) return SCOUP_OK;
  drop_graph(p);
  for (cudaStream_t s : p->lane_st) cudaStreamSynchronize(s);
  for (void* w : p->lane_ws) cudaFree(w);
  for (cudaStream_t s : p->lane_st) cudaStreamDestroy(s);
  for (cudaEvent_t ev : p->join_ev) cudaEventDestroy(ev);
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  if (p->cap_st) cudaStreamDestroy(p->cap_st);
  if (p->stats_dev) cudaFree(p->stats_dev);
  drain_release(&p->drain);
  delete p;
  return SCOUP_OK;
}

}  // extern "C"
