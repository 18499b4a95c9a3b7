// drain.cu -- the batched uplift as chunks of views, each chunk composited by
// one persistent tile launch (Sec. 4.2, Eq. 5 and Eq. 6 per scene; the
// batching itself has no counterpart in the paper).
//
// The views of all scenes are interleaved (view r of every scene, then view
// r + 1, ...) and cut into chunks of `chunk` views.  A chunk runs on one of
// `lanes` streams: each of its views is projected and binned into a view part
// of its own (records, depth, rectangles, tile lists and a header holding the
// view's depth range and counters); then one launch of the drain kernel
// composites every (view, tile) item of the chunk, its CTAs taking items from
// the lane's atomic counter (cleared before each drain; no CTA waits on
// another); then a merge kernel adds the views' counters into their scenes'
// headers (run_chunk, api.cu, shared with scoup_uplift's chunked form).
// Chunk c uses the view parts of lane c % lanes, so the projection and
// binning of one lane's chunk overlap the compositing of another's.  Every
// scene is set up once before the first chunk (header, accumulator,
// Morton-ordered copy, codes cut to K entries) and gets its Top-K after the
// last.  The schedule stays on the host: the chunk's views reach the kernels
// through their launch parameters.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "drain.cuh"

namespace scoup {
namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int kMaxParts = 64;

struct InitArgs {
  DrainViewInit part[kMaxParts];
  int max_tiles;
};

// Resets view parts before their first use: headers (counters, status, the
// depth range of every slot) and the binning counters.
__global__ void view_init_kernel(const __grid_constant__ InitArgs a) {
  const DrainViewInit& v = a.part[blockIdx.y];
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0) {
    WsHeader h = {};
    for (int q = 0; q < 4; ++q) { h.drange[q][0] = 0xffffffffu; h.drange[q][1] = 0u; }
    *v.hdr = h;
  }
  for (int t = t0; t <= a.max_tiles; t += stride) { v.tile_count[t] = 0u; v.tile_glob[t] = 0u; }
  for (int t = t0; t < kDepthBuckets; t += stride) v.dhist[t] = 0u;
}

struct MergeArgs {
  WsHeader* view[kMaxDrainJobs];
  WsHeader* scene[kMaxDrainJobs];
  int n;
};

// After a chunk's drain: adds each view's counters into its scene's header
// and clears them for the view part's next use.
__global__ void view_merge_kernel(const __grid_constant__ MergeArgs a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  WsHeader* v = a.view[j];
  WsHeader* s = a.scene[j];
  atomicAdd(&s->visible, v->visible);
  atomicAdd(&s->duplicates, v->duplicates);
  atomicAdd(&s->evaluated, v->evaluated);
  atomicAdd(&s->contributions, v->contributions);
  atomicAdd(&s->flushes, v->flushes);
  atomicAdd(&s->atomics, v->atomics);
  atomicAdd(&s->listed, v->listed);
  atomicAdd(&s->split_windows, v->split_windows);
  atomicMax(&s->max_dups_view, v->max_dups_view);
  if (v->status) atomicOr(&s->status, v->status);
  v->visible = v->duplicates = v->evaluated = v->contributions = 0ull;
  v->flushes = v->atomics = v->listed = v->split_windows = 0ull;
  v->max_dups_view = 0;
  v->status = 0;
}

}  // namespace

cudaError_t launch_view_init(const DrainViewInit* parts, int nparts, int max_tiles, cudaStream_t st) {
  for (int q0 = 0; q0 < nparts; q0 += kMaxParts) {
    InitArgs a;
    memset(&a, 0, sizeof(a));
    const int np = std::min(kMaxParts, nparts - q0);
    for (int q = 0; q < np; ++q) a.part[q] = parts[q0 + q];
    a.max_tiles = max_tiles;
    const int gx = std::min(64, (max_tiles + 1 + 255) / 256);
    view_init_kernel<<<dim3(gx, np), 256, 0, st>>>(a);
    g_launches += 1;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_view_merge(const TileJob* jobs, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (njobs > kMaxDrainJobs) return cudaErrorInvalidValue;
  MergeArgs m;
  memset(&m, 0, sizeof(m));
  m.n = njobs;
  for (int j = 0; j < njobs; ++j) {
    m.view[j] = jobs[j].hdr;
    m.scene[j] = jobs[j].scene_hdr;
  }
  view_merge_kernel<<<(njobs + 63) / 64, 64, 0, st>>>(m);
  g_launches += 1;
  return cudaGetLastError();
}

namespace {

void release_aux(DrainLayout* d) {
  for (cudaStream_t s : d->aux) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : d->aux_fork) cudaEventDestroy(e);
  for (cudaEvent_t e : d->aux_join) cudaEventDestroy(e);
  d->aux.clear();
  d->aux_fork.clear();
  d->aux_join.clear();
}

}  // namespace

void drain_release(DrainLayout* d) {
  release_aux(d);
  if (d->mem) cudaFree(d->mem);
  *d = DrainLayout();
}

static_assert(SCOUP_MAX_CHUNK_VIEWS <= kMaxDrainJobs, "a chunk's views fit one drain launch");

int drain_prepare(DrainLayout* d, const std::vector<scoup_batch_item>& items, const std::vector<int64_t>& max_dups,
                  int C, int K, int accum_mode, int chunk, int lanes, int sample) {
  if (chunk < 1 || lanes < 1) return set_error(SCOUP_ERR_INVALID_ARG, "chunk and lanes must be >= 1");
  const int B = (int)items.size();
  const bool compensated = (accum_mode & SCOUP_ACCUM_COMPENSATED) != 0;
  // views of every scene (all, or an evenly spaced sample) and the sizes
  std::vector<std::vector<int>> views(B);
  int64_t n_max = 0, dups_max = 1;
  int max_tiles = 1, rounds = 0;
  size_t scene_bytes = 0;
  for (int b = 0; b < B; ++b) {
    const scoup_batch_item& it = items[b];
    int mt = 1;
    int rc = check_scene_views(&it.scene, it.cams, it.V, &mt);
    if (rc) return rc;
    if (it.s < 1 || it.s > 1024) return set_error(SCOUP_ERR_INVALID_ARG, "batch item: s outside [1, 1024]");
    if (it.R_total < 0) return set_error(SCOUP_ERR_INVALID_ARG, "batch item: R_total < 0");
    if (it.V > 0 && (!it.region_maps || !it.map_offsets))
      return set_error(SCOUP_ERR_INVALID_ARG, "batch item: region maps are NULL");
    if (it.V > 0 && it.R_total > 0 && (!it.code_idx || !it.code_val))
      return set_error(SCOUP_ERR_INVALID_ARG, "batch item: code table is NULL");
    if (it.scene.n > 0 && !it.accum) return set_error(SCOUP_ERR_INVALID_ARG, "batch item: accum is NULL");
    if ((it.topk_idx == nullptr) != (it.topk_val == nullptr))
      return set_error(SCOUP_ERR_INVALID_ARG, "batch item: topk_idx and topk_val must both be given or both be NULL");
    for (int v = 0; v < it.V; ++v)
      if (it.map_offsets[v] < 0) return set_error(SCOUP_ERR_INVALID_ARG, "batch item: map_offsets < 0");
    const int take = (sample > 0 && sample < it.V) ? sample : it.V;
    for (int k = 0; k < take && it.scene.n > 0; ++k) views[b].push_back((int)((int64_t)k * it.V / take));
    rounds = std::max(rounds, (int)views[b].size());
    n_max = std::max(n_max, it.scene.n);
    max_tiles = std::max(max_tiles, mt);
    dups_max = std::max(dups_max, max_dups[b] + 1);
    const int64_t code_rows_k = it.s > K ? (int64_t)it.R_total * K : 0;
    scene_bytes += align_up(uplift_scene_part_bytes(it.scene.n, code_rows_k));
  }
  // chunks: view r of every scene, then view r + 1, ...
  std::vector<std::pair<int, int>> order;
  for (int r = 0; r < rounds; ++r)
    for (int b = 0; b < B; ++b)
      if (r < (int)views[b].size()) order.push_back({b, views[b][r]});
  const int njobs = (int)order.size();
  const int nchunks = (njobs + chunk - 1) / chunk;
  const int nparts = lanes * chunk;
  const size_t part_bytes = align_up(uplift_view_part_bytes(n_max, max_tiles));
  const size_t keys_bytes = align_up(sizeof(unsigned long long) * (size_t)dups_max);
  const size_t hdr_bytes = align_up(sizeof(WsHeader));
  const size_t need = scene_bytes + (size_t)nparts * (hdr_bytes + part_bytes + keys_bytes) +
                      align_up(sizeof(unsigned) * (size_t)lanes);
  cudaError_t e;
  if ((int)d->aux.size() != lanes) {
    release_aux(d);
    for (int l = 0; l < lanes; ++l) {
      cudaStream_t s = nullptr;
      cudaEvent_t f = nullptr, j = nullptr;
      if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) != cudaSuccess) {
        if (s) cudaStreamDestroy(s);
        if (f) cudaEventDestroy(f);
        release_aux(d);
        return set_error(SCOUP_ERR_CUDA, "chunked batch: streams");
      }
      d->aux.push_back(s);
      d->aux_fork.push_back(f);
      d->aux_join.push_back(j);
    }
  }
  if (need > d->bytes) {
    if ((e = cudaDeviceSynchronize()) != cudaSuccess)  // a run still in flight may use the old memory
      return set_error(SCOUP_ERR_CUDA, cudaGetErrorString(e));
    if (d->mem) cudaFree(d->mem);
    d->mem = nullptr;
    d->bytes = 0;
    if ((e = cudaMalloc(&d->mem, need)) != cudaSuccess) {
      d->mem = nullptr;
      return set_error(SCOUP_ERR_OOM, "chunked batch: device memory");
    }
    d->bytes = need;
  }
  d->chunk = 0;  // no layout until this one is complete
  d->max_tiles = max_tiles;
  char* p = (char*)d->mem;
  size_t off = 0;
  d->scene.assign(B, UpliftWs());
  d->fci.assign(B, nullptr);
  d->fcv.assign(B, nullptr);
  for (int b = 0; b < B; ++b) {
    const int64_t code_rows_k = items[b].s > K ? (int64_t)items[b].R_total * K : 0;
    off += align_up(carve_scene_part(p + off, items[b].scene.n, code_rows_k, &d->scene[b], &d->fci[b], &d->fcv[b]));
    if (code_rows_k == 0) { d->fci[b] = nullptr; d->fcv[b] = nullptr; }
  }
  d->view.assign(nparts, UpliftWs());
  d->init.assign(nparts, DrainViewInit());
  for (int q = 0; q < nparts; ++q) {
    UpliftWs& w = d->view[q];
    w.hdr = (WsHeader*)(p + off);
    off += hdr_bytes;
    off += carve_view_part(p + off, n_max, max_tiles, &w);
    w.keys = (unsigned long long*)(p + off);
    w.dup_capacity = dups_max;
    off += keys_bytes;
    d->init[q] = DrainViewInit{w.hdr, w.tile_count, w.tile_glob, w.dhist};
  }
  d->counters_dev = (unsigned*)(p + off);
  // the schedule
  d->jobs.assign(njobs, TileJob());
  d->job_view_part.assign(njobs, 0);
  d->chunk_begin.assign(nchunks + 1, njobs);
  d->tile0.assign(std::max(njobs, 1), 0u);
  for (int c = 0; c < nchunks; ++c) {
    d->chunk_begin[c] = c * chunk;
    uint32_t items_c = 0;
    for (int j = c * chunk; j < std::min(njobs, (c + 1) * chunk); ++j) {
      const int b = order[j].first, v = order[j].second;
      const scoup_batch_item& it = items[b];
      const int q = (c % lanes) * chunk + (j - c * chunk);
      const UpliftWs& w = d->view[q];
      TileJob& J = d->jobs[j];
      J.cam = camera_args(it.cams[v]);
      const bool cut = d->fci[b] != nullptr;
      J.lc = LevelCodes();
      J.lc.L = 1;
      J.lc.s_tot = cut ? K : it.s;
      J.lc.rmap[0] = it.region_maps + it.map_offsets[v];
      J.lc.ci[0] = cut ? d->fci[b] : it.code_idx;
      J.lc.cv[0] = cut ? d->fcv[b] : it.code_val;
      J.lc.s[0] = J.lc.s_tot;
      J.lc.R[0] = it.R_total;
      J.proj = w.proj;
      J.keys = w.keys;
      J.tile_start = w.tile_start;
      J.accum = it.accum;
      J.comp = compensated ? it.accum + (size_t)it.scene.n * (size_t)C : nullptr;
      J.hdr = w.hdr;
      J.scene_hdr = d->scene[b].hdr;
      J.slot = (c / lanes) & 1;
      J.C = C;
      J.tiles = J.cam.gx * J.cam.gy;
      J.scene = b;
      d->job_view_part[j] = q;
      d->tile0[j] = items_c;
      items_c += (uint32_t)J.tiles;
    }
  }
  d->chunk = chunk;
  d->lanes = lanes;
  d->sample = sample;
  return SCOUP_OK;
}

int drain_enqueue(DrainLayout* d, const std::vector<scoup_batch_item>& items, int C, int K, int accum_mode,
                  int warp_w, const cudaStream_t* lane_st, const cudaEvent_t* join_ev, cudaEvent_t fork_ev,
                  WsHeader* stats_dev, cudaStream_t st) {
  const int B = (int)items.size();
  const bool compensated = (accum_mode & SCOUP_ACCUM_COMPENSATED) != 0;
  const int nparts = d->lanes * d->chunk;
  const int nchunks = std::max(0, (int)d->chunk_begin.size() - 1);
  auto fail_cuda = [](cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof(buf), "chunked batch, %s: %s", where, cudaGetErrorString(e));
    return set_error(SCOUP_ERR_CUDA, buf);
  };
  cudaError_t e;
  // every scene: header, accumulator, codes cut to K entries, Morton-ordered copy
  for (int b = 0; b < B; ++b) {
    const scoup_batch_item& it = items[b];
    const UpliftWs& sw = d->scene[b];
    const int64_t n = it.scene.n;
    if ((e = cudaMemsetAsync(sw.hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return fail_cuda(e, "header");
    if (n == 0) continue;
    if (!(accum_mode & SCOUP_ACCUM_CONTINUE) &&
        (e = cudaMemsetAsync(it.accum, 0, sizeof(float) * (size_t)n * (size_t)C * (compensated ? 2 : 1), st)) !=
            cudaSuccess)
      return fail_cuda(e, "accumulator");
    if (d->fci[b] && it.R_total > 0 &&
        (e = launch_code_topk(it.code_idx, it.code_val, it.R_total, it.s, K, d->fci[b], d->fcv[b], st)) != cudaSuccess)
      return fail_cuda(e, "code top-k");
    if (it.V > 0 && (e = launch_reorder(it.scene, sw, st)) != cudaSuccess) return fail_cuda(e, "reorder");
  }
  // the view parts
  if (nparts > 0 && (e = launch_view_init(d->init.data(), nparts, d->max_tiles, st)) != cudaSuccess)
    return fail_cuda(e, "init");
  // chunks on the lanes
  const int used = std::min(d->lanes, nchunks);
  if (used > 0 && (e = cudaEventRecord(fork_ev, st)) != cudaSuccess) return fail_cuda(e, "fork");
  for (int l = 0; l < used; ++l)
    if ((e = cudaStreamWaitEvent(lane_st[l], fork_ev, 0)) != cudaSuccess) return fail_cuda(e, "fork wait");
  int rc = SCOUP_OK;
  std::vector<UpliftWs> vw;
  std::vector<const scoup_scene*> vs;
  for (int c = 0; c < nchunks && rc == SCOUP_OK; ++c) {
    const int lane = c % d->lanes;
    const int j0 = d->chunk_begin[c], j1 = d->chunk_begin[c + 1];
    vw.clear();
    vs.clear();
    for (int j = j0; j < j1; ++j) {
      const TileJob& J = d->jobs[j];
      UpliftWs w = d->view[d->job_view_part[j]];
      w.sp = d->scene[J.scene].sp;
      w.cell = d->scene[J.scene].cell;
      w.cells_scratch = d->scene[J.scene].cells_scratch;
      vw.push_back(w);
      vs.push_back(&items[J.scene].scene);
    }
    const ChunkStreams cs{lane_st[lane], d->aux[lane], d->aux_fork[lane], d->aux_join[lane]};
    rc = run_chunk(d->jobs.data() + j0, d->tile0.data() + j0, j1 - j0, vw.data(), vs.data(), d->counters_dev + lane,
                   compensated, warp_w, cs);
  }
  // join even on an error, so that a capture in progress stays well formed
  for (int l = 0; l < used; ++l)
    if ((e = cudaEventRecord(join_ev[l], lane_st[l])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, join_ev[l], 0)) != cudaSuccess)
      if (rc == SCOUP_OK) rc = fail_cuda(e, "join");
  if (rc != SCOUP_OK) return rc;
  for (int b = 0; b < B; ++b) {
    const scoup_batch_item& it = items[b];
    const int64_t n = it.scene.n;
    if (it.topk_idx && n > 0 &&
        (e = launch_topk(it.accum, compensated ? it.accum + (size_t)n * (size_t)C : nullptr, n, C, K, it.topk_idx,
                         it.topk_val, nullptr, st, C)) != cudaSuccess)
      return fail_cuda(e, "top-k");
    if (stats_dev && (e = cudaMemcpyAsync(stats_dev + b, d->scene[b].hdr, sizeof(WsHeader), cudaMemcpyDeviceToDevice,
                                          st)) != cudaSuccess)
      return fail_cuda(e, "stats copy");
  }
  return SCOUP_OK;
}

}  // namespace scoup
