// drain.cuh -- the chunked batched uplift (drain.cu), driven by batch.cu.
#pragma once

#include <vector>

#include "scoup_internal.cuh"

namespace scoup {

// Pointers of one view part that are reset before a batch.
struct DrainViewInit {
  WsHeader* hdr;
  uint32_t* tile_count;
  uint32_t* tile_glob;
  uint32_t* dhist;
};

// Streams of one chunk lane: the lane's stream and a second one that
// projects and bins the odd views of a chunk (null: all on the lane's stream),
// with the events that fork it from and join it back into the lane's stream.
struct ChunkStreams {
  cudaStream_t ls, as;
  cudaEvent_t fork, join;
  cudaEvent_t before_drain = nullptr;  // if set: the drain waits for it (staged region maps)
  cudaEvent_t after_drain = nullptr;   // if set: recorded once the drain and merge are enqueued
};

// One chunk of njobs <= kMaxDrainJobs views (HOST arrays): projection and
// binning of each view into views[j] (its view part, with the scene copy of
// *scenes[j]), one drain launch over every (view, tile) item (tile0 as for
// launch_uplift_drain; *counter is cleared first), then the merge of the
// views' counters into their scenes' headers (api.cu).
int run_chunk(const TileJob* jobs, const uint32_t* tile0, int njobs, const UpliftWs* views,
              const scoup_scene* const* scenes, unsigned* counter, bool compensated, int warp_w,
              const ChunkStreams& cs);
// Resets view parts before their first use (headers, binning counters).
cudaError_t launch_view_init(const DrainViewInit* parts, int nparts, int max_tiles, cudaStream_t st);
// Adds each job's view counters into its scene header and clears them.
cudaError_t launch_view_merge(const TileJob* jobs, int njobs, cudaStream_t st);

// Device memory and the chunk schedule of the chunked form for one plan.
struct DrainLayout {
  int chunk = 0, lanes = 0, sample = -1;  // the configuration the layout was built for
  int max_tiles = 1;
  void* mem = nullptr;
  size_t bytes = 0;
  std::vector<UpliftWs> scene;         // per scene: its header and Morton-ordered copy
  std::vector<int32_t*> fci;           // per scene: codes cut to K entries (s > K) or null
  std::vector<float*> fcv;
  std::vector<UpliftWs> view;          // [lanes * chunk] view parts, each with its own header
  std::vector<TileJob> jobs;           // chunk-major: jobs[chunk_begin[c] .. chunk_begin[c + 1])
  std::vector<int> chunk_begin;        // [nchunks + 1]
  std::vector<int> job_view_part;      // view part of each job
  std::vector<uint32_t> tile0;        // per job: its first item within its chunk
  unsigned* counters_dev = nullptr;    // [lanes]: the drain counter of each lane
  std::vector<DrainViewInit> init;     // [lanes * chunk]
  // per lane: a second stream projecting and binning the odd views of the
  // lane's chunk, forked from and joined back into the lane's stream
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> aux_fork, aux_join;
};

// Builds (or rebuilds) the layout for `chunk` views per chunk on `lanes`
// streams over the items (every view, or `sample` evenly spaced views per
// scene when sample > 0); max_dups[b] is scene b's largest per-view pair
// count.  Creates the lanes' second streams and, when the layout outgrows the
// memory it has, synchronises the device and reallocates: never while a
// stream is capturing.
int drain_prepare(DrainLayout* d, const std::vector<scoup_batch_item>& items, const std::vector<int64_t>& max_dups,
                  int C, int K, int accum_mode, int chunk, int lanes, int sample);

// Enqueues the batch: set-up on `st`, chunks on the lane streams (forked from
// and joined back into `st`), Top-K on `st`; stats_dev (or null) receives a
// copy of each scene's header.  Capturable.
int drain_enqueue(DrainLayout* d, const std::vector<scoup_batch_item>& items, int C, int K, int accum_mode,
                  int warp_w, const cudaStream_t* lane_st, const cudaEvent_t* join_ev, cudaEvent_t fork_ev,
                  WsHeader* stats_dev, cudaStream_t st);

void drain_release(DrainLayout* d);

}  // namespace scoup
