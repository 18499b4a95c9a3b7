/*
 * scoup.h -- C ABI of the GB300 (sm_103a) SCOUP sparse code uplift library.
 *
 * SCOUP (Sparse Code Uplifting) lifts per-region sparse codebook codes of
 * 2D views onto the Gaussians of a pretrained 3D Gaussian Splatting scene,
 * keeps a Top-K code per Gaussian, and renders those codes back to 2D.
 *
 * Conventions
 *  - Every entry point returns an int status: SCOUP_OK (0) or a negative
 *    SCOUP_ERR_* code; scoup_last_error() then holds a message for the
 *    calling thread.  Nothing aborts or exits.
 *  - Array pointers are DEVICE pointers owned by the caller (contiguous,
 *    row-major, 16-byte aligned where noted); small descriptors (scene,
 *    cameras, offsets) are HOST structs/arrays.  The library never frees
 *    caller memory and allocates no device memory of its own on these
 *    paths: scratch is the caller's `workspace`.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream) and is complete when the stream is.  Calls
 *    do not synchronise, except those that take a host `scoup_stats*`
 *    (non-NULL) or read back sizes, as documented per function.
 *  - Errors detected on the device (workspace capacity exceeded, invalid
 *    region or atom ids) are recorded in the workspace status word and
 *    returned by the next synchronising call (scoup_read_stats, or the call
 *    itself when it was given `stats`).
 */
#ifndef SCOUP_H
#define SCOUP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCOUP_OK 0
#define SCOUP_ERR_INVALID_ARG (-1)   /* host-side argument validation failed */
#define SCOUP_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define SCOUP_ERR_OOM (-3)           /* workspace smaller than required */
#define SCOUP_ERR_CAPACITY (-4)      /* device: tile-list capacity exceeded */
#define SCOUP_ERR_DEVICE_CHECK (-5)  /* device: region/atom id out of range */
#define SCOUP_ERR_TIMEOUT (-6)       /* device: a bounded wait in a tensor-core pipeline gave up */

/* Gaussians of a 3DGS scene (paper Sec. 3): means mu_i, linear scales s_i
 * (exp of the stored log-scales), unit quaternions q_i in (w, x, y, z)
 * order (normalised again inside), opacities o_i in (0, 1] after the
 * sigmoid.  Device pointers, float32, row-major [n,3], [n,3], [n,4], [n]. */
typedef struct scoup_scene {
  int64_t n;
  const float* means;
  const float* scales;
  const float* quats;
  const float* opacity;
} scoup_scene;

/* Pinhole camera: world->camera 3x4 row-major [R | t] with camera x right,
 * y down, z forward; focal lengths and principal point in pixels; pixel
 * (x, y) is sampled at image point (x + 0.5, y + 0.5). */
typedef struct scoup_camera {
  float viewmat[12];
  float fx, fy, cx, cy;
  int32_t width, height;
} scoup_camera;

/* Counters of one uplift or render call (summed over its views). */
typedef struct scoup_stats {
  int64_t visible;          /* (Gaussian, view) pairs that survive culling */
  int64_t duplicates;       /* (Gaussian, tile) pairs of the 3DGS tile rectangles */
  int64_t evaluated_pairs;  /* (pixel, Gaussian) pairs examined while the pixel was active */
  int64_t contributions;    /* accepted pairs: alpha >= 1/255, before the transmittance stop */
  int64_t flushes;          /* (Gaussian, tile, region) partial sums flushed to the accumulator */
  int64_t atomics;          /* global accumulator atomics issued */
  int64_t listed;           /* (Gaussian, tile) pairs kept after the exact alpha-reach test */
  int32_t status;           /* SCOUP_OK or the first device-side error */
  int32_t max_dups_view;    /* largest per-view duplicate count seen */
  int64_t split_windows;    /* ordering windows cut out of one depth bucket that held more
                               keys than a window (ties in depth, fronto-parallel sheets) */
} scoup_stats;

const char* scoup_version(void);
const char* scoup_last_error(void);

/* ------------------------------------------------------------------ */
/* Uplift (paper Sec. 4.2, Eq. 5 and Eq. 6, Algorithm 1)                */
/* ------------------------------------------------------------------ */

/* Bytes of workspace for scoup_uplift on scenes of up to n Gaussians, views
 * of up to max_width x max_height pixels and up to dup_capacity
 * (Gaussian, tile) pairs per view.  scoup_uplift runs even and odd views in
 * two pipelines (the second on a stream the library owns, joined back into
 * the caller's stream) when the workspace holds two sets of per-view buffers;
 * this size provides them; a workspace too small for two runs one.
 * Returns 0 on invalid arguments. */
size_t scoup_uplift_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                   int64_t dup_capacity);

/* Exact per-view (Gaussian, tile) pair counts: projects every view and
 * writes the largest count to *max_dups (host).  Synchronises `stream`.
 * workspace may be sized with any dup_capacity >= 0. */
int scoup_uplift_plan(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                      void* workspace, size_t ws_bytes, int64_t* max_dups, void* stream);

#define SCOUP_ACCUM_CONTINUE 1    /* accum_mode: add to the accumulator instead of zeroing it */
#define SCOUP_ACCUM_COMPENSATED 2 /* accum_mode: compensated (TwoSum) FP32 accumulation */
#define SCOUP_UPLIFT_CHUNKED 4    /* accum_mode: composite the views in chunks (see scoup_uplift) */

/* Sparse coefficient uplift.  For every view v (cams[v], host array of V),
 * rasterizes the scene with standard 3DGS compositing (Sec. 3, Eq. 2) and
 * adds, for every accepted (pixel p, Gaussian i) pair with weight
 * e = alpha * T, c * e to accum[i][j] for every code entry (j, c) of the
 * region of p (Eq. 5 without Z_i, which Eq. 6 makes redundant).  Then, if
 * topk_idx != NULL, writes per Gaussian the K largest positive entries of
 * its accumulator row (ties to the lower atom index) divided by their sum
 * (Eq. 6), padded with (-1, 0).
 *
 *  region_maps  int32, views packed back to back; view v occupies
 *               [map_offsets[v], map_offsets[v] + H_v*W_v), row-major; each
 *               value is a row of the code table or -1 (unlabelled pixel:
 *               occludes, contributes nothing).
 *  map_offsets  HOST int64 [V] element offsets into region_maps.
 *  R_total      number of code-table rows (region ids must be < R_total).
 *  code_idx     int32 [R_total, s] atom ids (< C) or -1 padding.
 *  code_val     float32 [R_total, s] nonnegative coefficients (Eq. 4).
 *               If s > K, each code's K largest entries are used (Alg. 1).
 *  accum        float32 [n, C] row-major accumulator (caller-owned); with
 *               SCOUP_ACCUM_COMPENSATED, float32 [2, n, C]: the running sums
 *               followed by their compensation terms (value = sum + term).
 *  accum_mode   bit flags.  Without SCOUP_ACCUM_CONTINUE accum is zeroed
 *               first; with it the call adds to the current contents (resume
 *               an uplift whose views were split over several calls).
 *               SCOUP_ACCUM_COMPENSATED: every FP32
 *               addition into the per-tile partials and into accum carries
 *               its exact rounding error (TwoSum) into a compensation term,
 *               as does the product code value x weight; Top-K ranks
 *               sum + term.  Slower (one more atomic per update).
 *               SCOUP_UPLIFT_CHUNKED (the fast form; single level): the
 *               views are cut into chunks of 8 on two lanes (streams); each
 *               view of a chunk is projected and binned into a view part of
 *               its own, then ONE persistent tile launch composites every
 *               (view, tile) item of the chunk, its CTAs taking items from
 *               an atomic counter.  Same results up to the order of FP32
 *               atomic additions; same counters.  The workspace must then be
 *               sized by scoup_uplift_chunked_workspace_size (16 view parts).
 *  topk_idx     int32 [n, K] or NULL (accumulate only); topk_val float32 [n, K].
 *  workspace    device scratch of ws_bytes >= scoup_uplift_workspace_size()
 *               (scoup_uplift_chunked_workspace_size() with SCOUP_UPLIFT_CHUNKED;
 *               a smaller one is refused with SCOUP_ERR_OOM before any work).
 *  stats        HOST scoup_stats* or NULL; when given, the call synchronises
 *               `stream` and returns the device status.
 * Limits: 1 <= K <= C <= 1024, 1 <= s <= 1024, V >= 0, n >= 0 (n = 0 and V = 0
 * are valid and produce empty / padded outputs).
 *
 * Dense feature uplift (Eq. 3, the formulation sparse coding replaces) is the
 * same call with each region's D-dimensional feature as its code: C = s = K =
 * D + 1, code_idx[r] = (0, 1, ..., D), code_val[r] = (F_r, 1), topk_idx NULL;
 * then f_i = accum[i][0:D] / accum[i][D] (accum[i][D] = Z_i). */
int scoup_uplift(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                 const int32_t* region_maps, const int64_t* map_offsets, int32_t R_total,
                 const int32_t* code_idx, const float* code_val, int32_t s, int32_t C, int32_t K,
                 float* accum, int32_t accum_mode, int32_t* topk_idx, float* topk_val,
                 void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream);

/* Workspace bytes for scoup_uplift with SCOUP_UPLIFT_CHUNKED: the scene part
 * and 2 x 8 view parts, each holding dup_capacity (Gaussian, tile) keys (the
 * largest per-view pair count, scoup_uplift_plan).  0 on invalid arguments. */
size_t scoup_uplift_chunked_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                           int64_t dup_capacity);

/* Workspace bytes for scoup_uplift_host_maps: a staging ring of 4 view maps
 * of max_width x max_height int32 entries, then a scoup_uplift workspace
 * (scoup_uplift_workspace_size with the same arguments).  0 on invalid
 * arguments. */
size_t scoup_uplift_host_maps_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                             int64_t dup_capacity);

/* Workspace bytes for scoup_uplift_host_maps with SCOUP_UPLIFT_CHUNKED: a
 * staging ring of 16 view maps (one per view part) of max_width x max_height
 * int32 entries, then the chunked layout (scoup_uplift_chunked_workspace_size
 * with the same arguments).  0 on invalid arguments. */
size_t scoup_uplift_host_maps_chunked_workspace_size(int64_t n, int32_t max_width, int32_t max_height,
                                                     int64_t dup_capacity);

/* scoup_uplift with the region maps in HOST memory (pinned for the copies to
 * run asynchronously): view v's map is copied to a ring slot in the workspace
 * on a library copy stream while earlier views compute, and only view v's
 * tile pass waits for it (its projection and binning do not read the map).
 * With SCOUP_UPLIFT_CHUNKED the maps of a chunk are copied while the lane's
 * previous chunk composites, and the chunk's drain waits for them (workspace:
 * scoup_uplift_host_maps_chunked_workspace_size).
 * Results equal scoup_uplift on the same maps up to the order of the FP32
 * atomic additions (as two scoup_uplift runs do); counters are equal.  The copies
 * follow the work already on `stream` and the call's work is joined back
 * into it.  Single level; not for graph capture (the copy stream is not
 * forked from a capturing stream).  Other arguments as scoup_uplift;
 * workspace >= scoup_uplift_host_maps_workspace_size(...) bytes, sized with
 * max_width / max_height covering every view. */
int scoup_uplift_host_maps(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                           const int32_t* host_region_maps, const int64_t* map_offsets, int32_t R_total,
                           const int32_t* code_idx, const float* code_val, int32_t s, int32_t C, int32_t K,
                           float* accum, int32_t accum_mode, int32_t* topk_idx, float* topk_val,
                           void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream);

/* One semantic level of a multi-level uplift: the region maps of every view
 * (packed as for scoup_uplift, same map_offsets for all levels) and the
 * level's code table. */
typedef struct scoup_level {
  const int32_t* region_maps;  /* DEVICE int32, -1 = unlabelled at this level */
  int32_t R_total;
  const int32_t* code_idx;     /* DEVICE [R_total, s] */
  const float* code_val;       /* DEVICE [R_total, s] */
  int32_t s;
} scoup_level;

/* Uplift of L <= 3 semantic levels in one pass (the paper runs its three SAM
 * levels as independent uplifts, Sec. 5.1; the compositing weights e do not
 * depend on the level, so one rasterisation serves them all).  Results are
 * those of L scoup_uplift calls, one per level:
 *  accum     DEVICE float32 [n, L*C]; level l in columns [l*C, (l+1)*C)
 *            ([2, n, L*C] with SCOUP_ACCUM_COMPENSATED).
 *  topk_idx, topk_val  DEVICE [L, n, K] or NULL.
 * Limits as for scoup_uplift, and per level s <= K, sum of s <= 64,
 * R_total < 2^21 - 1.  Workspace and stats as for scoup_uplift.
 * Rendering all levels at once is scoup_render with C' = L*C, K' = L*K and
 * each Gaussian's codes of level l concatenated with atom ids offset by l*C:
 * out_codes[p][l*C + j] is level l's rendered code. */
int scoup_uplift_levels(const scoup_scene* scene, const scoup_camera* cams, int32_t V, const int64_t* map_offsets,
                        const scoup_level* levels, int32_t L, int32_t C, int32_t K, float* accum,
                        int32_t accum_mode, int32_t* topk_idx, float* topk_val, void* workspace, size_t ws_bytes,
                        scoup_stats* stats, void* stream);

/* Top-K + L1 normalisation (Eq. 6) of an accumulator accum[n, C] alone:
 * positive entries only, ordered by (value desc, atom index asc), divided by
 * the sum of the kept values; rows without positive entries give (-1, 0). */
int scoup_topk(const float* accum, int64_t n, int32_t C, int32_t K, int32_t* topk_idx,
               float* topk_val, void* stream);

/* Synchronises `stream` and reads the counters and status of the last call
 * that used this workspace. */
int scoup_read_stats(const void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream);

/* ------------------------------------------------------------------ */
/* Sparse coefficient rendering (paper Sec. 4.3, Eq. 7)                 */
/* ------------------------------------------------------------------ */

/* Renders one view: What(p) = sum_i e_i(p) w^_i over the Gaussians in front
 * to back order with the same compositing as scoup_uplift (Eq. 2), where
 * w^_i is Gaussian i's K-sparse code (topk_idx[i][k] < C or -1 padding,
 * topk_val[i][k]).  The result is the dense, unnormalised C-vector per pixel.
 *  out_codes  [H, W, C] row-major (every pixel written): float32 with
 *             out_dtype 0, bf16 (round to nearest even) with out_dtype 1 --
 *             the input scoup_decode takes without conversion.
 * Two kernels compute it.  For C <= 256 and K <= 16 the tile's codes are a
 * tensor-core contraction accumulated in FP32 (each weight and coefficient
 * carried as two bf16 parts: at most about 3 * 2^-16 relative error per product) and
 * rounded to the output type once.  Wider rows (or SCOUP_RENDER_SIMT=1 in the
 * environment) take the SIMT kernel, which sums in FP32 in list order and,
 * with bf16 output, rounds after each window of 256 list entries (a pixel
 * spanning w windows: relative error at most w 2^-8, bf16 unit roundoff).
 *  out_T      float32 [H, W] final transmittance, or NULL.
 *  out_last   int32 [H, W]: number of front-to-back list entries up to and
 *             including the last contributor of the pixel, or NULL.
 *  workspace  as for scoup_uplift with one view (scoup_uplift_workspace_size
 *             with the camera's size).
 *  stats      HOST or NULL; when given, the call synchronises `stream`.
 * Limits: 1 <= K <= C <= 1024. */
int scoup_render(const scoup_scene* scene, const int32_t* topk_idx, const float* topk_val, int32_t K,
                 int32_t C, const scoup_camera* cam, void* out_codes, int32_t out_dtype, float* out_T,
                 int32_t* out_last, void* workspace, size_t ws_bytes, scoup_stats* stats, void* stream);

/* Workspace bytes for scoup_render_decode_fused on views of width x height:
 * the decode workspace, the view's bf16 rendered codes and a render
 * workspace (scoup_uplift_workspace_size with the same n, size and
 * dup_capacity).  Returns 0 on invalid arguments. */
size_t scoup_render_decode_workspace_size(int64_t n, int32_t width, int32_t height, int32_t C, int32_t D,
                                          int64_t dup_capacity);

/* Eq. 7 then Eq. 8 in one call: renders the view (scoup_render with bf16
 * codes) into the workspace and decodes those codes with the codebook
 * (scoup_decode with codes_dtype 1) on the same stream.  The results equal
 * the two separate calls bit for bit (the same kernels on the same values);
 * the rendered codes never reach a caller array.
 *  codebook    DEVICE float32 [C, D] row-major.
 *  features    DEVICE [H * W, D] row-major, float32 (out_dtype 0) or bf16
 *              (out_dtype 1), 16-byte aligned; feat_norm2 as in scoup_decode.
 *  out_T, out_last as in scoup_render (or NULL).
 *  workspace   DEVICE, >= scoup_render_decode_workspace_size(...) bytes.
 *  stats       HOST or NULL: the render's counters and the first nonzero
 *              status of either stage; when given, the call synchronises.
 * Limits: those of both calls (1 <= K <= C <= 1024, C a multiple of 8;
 * D a multiple of 16).  Why two kernels and not one: at C = 256 a tile's
 * FP32 codes take all 512 TMEM columns of the SM, the decode's 256 x 512
 * FP32 result would need as many again, and the bf16 code tile the decode
 * reads (128 KB) plus codebook stages leave no shared memory for the next
 * tile's walk, so a fused kernel would run the decode with the SM's walkers
 * idle; the separate persistent GEMM streams above 80% of the HBM copy rate. */
int scoup_render_decode_fused(const scoup_scene* scene, const int32_t* topk_idx, const float* topk_val, int32_t K,
                              int32_t C, const scoup_camera* cam, const float* codebook, int32_t D,
                              void* features, int32_t out_dtype, float* feat_norm2, float* out_T,
                              int32_t* out_last, void* workspace, size_t ws_bytes, scoup_stats* stats,
                              void* stream);

/* Gradient through scoup_render (derived from Eq. 2 and Eq. 7) for a loss
 * whose gradient with respect to the rendered codes is dL_dcodes (float32
 * [H, W, C]).  ADDS into the caller's arrays (zero them first for a fresh
 * gradient):
 *   d_topk_val[i][k] += sum_p e_i(p) dL_dcodes[p][topk_idx[i][k]]
 *   d_opacity[i]     += sum_p dalpha_i/do_i (T_i g.w^_i - S_after_i / (1 - alpha_i))
 * with S_after_i the sum of e_j g.w^_j over the contributors behind i and
 * dalpha/do = G_i(p) while o_i G_i(p) < 0.99, else 0.  Top-K indices and the
 * discrete compositing decisions are held fixed.  Transmittance is recomputed
 * (two front-to-back passes), nothing per pixel is stored between the calls.
 * Workspace and stats as for scoup_render.  Limits: 1 <= K <= min(C, 64). */
int scoup_render_backward(const scoup_scene* scene, const int32_t* topk_idx, const float* topk_val,
                          int32_t K, int32_t C, const scoup_camera* cam, const float* dL_dcodes,
                          float* d_topk_val, float* d_opacity, void* workspace, size_t ws_bytes,
                          scoup_stats* stats, void* stream);

/* Top-K + L1 normalisation (Eq. 6) as scoup_topk, fused with the entropy of
 * each row's coefficient distribution (the entropy analysis of Top-K
 * filtering): with p_l = w_l / sum w over the positive entries,
 * entropy[i] = -sum_l p_l log p_l (0 for a row with no positive entry).
 *  comp      DEVICE float32 [n, C] compensation terms of a compensated uplift
 *            (the second half of its accum), or NULL.
 *  entropy   DEVICE float32 [n].  Asynchronous. */
int scoup_topk_entropy(const float* accum, const float* comp, int64_t n, int32_t C, int32_t K, int32_t* topk_idx,
                       float* topk_val, float* entropy, void* stream);

/* Entropy filter: keeps the `keep` Gaussians of lowest entropy (ties to the
 * lower index) and clears the Top-K rows of all others to (-1, 0).
 *  entropy    DEVICE float32 [n] (e.g. from scoup_topk_entropy).
 *  topk_idx, topk_val  DEVICE [n, K], modified in place, or both NULL.
 *  keep_mask  DEVICE uint8 [n] (1 kept, 0 removed) or NULL.
 *  workspace  DEVICE, >= scoup_entropy_filter_workspace_size() bytes,
 *             16-byte aligned (overwritten).
 * Exact selection in 8 histogram passes; each pass's last CTA picks the next
 * digit on the device, so the call is asynchronous (enqueued on `stream`, no
 * synchronisation) and can be captured in a CUDA graph. */
size_t scoup_entropy_filter_workspace_size(void);
int scoup_entropy_filter(const float* entropy, int64_t n, int64_t keep, int32_t K, int32_t* topk_idx,
                         float* topk_val, uint8_t* keep_mask, void* workspace, size_t ws_bytes, void* stream);

/* Similarity and relevancy in one pass (App. B, Eq. 9): the cosine
 * similarity GEMM of scoup_similarity whose epilogue turns each pixel's row of
 * Q similarities straight into the relevancy of the Q - n_canon queries
 * against the n_canon canonical phrases (the first n_canon text vectors), as
 * scoup_relevancy would from scoup_similarity's output: the similarity matrix
 * never reaches memory.  Same features, feat_norm2, text, workspace (size
 * scoup_similarity_workspace_size(P, D, Q)) and rounding as scoup_similarity.
 *  Q          16 or 32 (one column tile); Q - n_canon a multiple of 4.
 *  alpha      > 0 (10 in the paper).
 *  R          DEVICE float32 [P, Q - n_canon], 16-byte aligned.
 * Results equal scoup_similarity followed by scoup_relevancy bit for bit.
 * Asynchronous. */
int scoup_similarity_relevancy(const void* features, int64_t P, int32_t D, const float* feat_norm2,
                               const float* text, int32_t Q, int32_t n_canon, float alpha, float* R,
                               void* workspace, size_t ws_bytes, void* stream);

/* Workspace bytes for scoup_decode_query. */
size_t scoup_decode_query_workspace_size(int64_t P, int32_t C, int32_t D, int32_t Q);

/* The codebook decode (Sec. 4.3, Eq. 8) with the text query of App. B in the
 * same tensor-core GEMM: F = What C is decoded as by scoup_decode (bf16
 * features, their squared norms), and the similarity of every row,
 *   s[p][q] = <F_p, t_q> / (|F_p| |t_q|)  (0 where |F_p| < 1e-12 or |t_q| = 0),
 * comes out of the same GEMM through the associativity
 * <What_p C, t_q> = <What_p, C t_q>: the Q columns G = C T^T (FP32 sums,
 * rounded to bf16) are a last 16- or 32-column unit of each 128-row block,
 * whose epilogue divides by |F_p| (the norm of the row's rounded features,
 * summed in the same CTA over the block's columns) and |t_q| (FP32, of the
 * text as given).  The features therefore never have to be read back, and
 * need not be stored at all.
 *  codes, codes_dtype, P, C, codebook, D   as for scoup_decode.
 *  text       DEVICE float32 [Q, D]; Q is 16 or 32 (pad with zero rows:
 *             their similarity is 0).
 *  n_canon    0: out receives the similarities [P, Q].  1 <= n_canon < Q:
 *             out receives the relevancy (App. B, Eq. 9, temperature alpha
 *             > 0) of the Q - n_canon queries (text rows n_canon..Q-1)
 *             against the n_canon canonical phrases (rows 0..n_canon-1),
 *             [P, Q - n_canon]; Q - n_canon a multiple of 4.
 *  features   DEVICE bf16 [P, D] or NULL (the features are then not written).
 *  feat_norm2 DEVICE float32 [P] or NULL: squared norms of the rounded rows.
 *  out        DEVICE float32, 16-byte aligned.
 *  workspace  DEVICE, >= scoup_decode_query_workspace_size(P, C, D, Q) bytes.
 * The similarity's numerator rounds What and G (not F) to bf16, so it is not
 * bit-equal to scoup_decode followed by scoup_similarity; both lie within the
 * bf16 bounds of the exact FP64 value.  Asynchronous; errors as for
 * scoup_decode. */
int scoup_decode_query(const void* codes, int32_t codes_dtype, int64_t P, int32_t C, const float* codebook,
                       int32_t D, const float* text, int32_t Q, int32_t n_canon, float alpha, void* features,
                       float* feat_norm2, float* out, void* workspace, size_t ws_bytes, void* stream);

/* Relevancy score of text queries (App. B, Eq. 9):
 *   R[p][q] = min_k exp(a s_q) / (exp(a s_q) + exp(a s_k))
 * from the similarities sim [P, ncols] (scoup_similarity output) whose first
 * n_canon columns are the canonical phrases and the other ncols - n_canon the
 * queries; a = alpha > 0 (10 in the paper).  R DEVICE float32 [P, ncols - n_canon].
 * Asynchronous. */
int scoup_relevancy(const float* sim, int64_t P, int32_t ncols, int32_t n_canon, float alpha, float* R,
                    void* stream);

/* ------------------------------------------------------------------ */
/* Batched uplift: many scenes with their own views, one graph launch   */
/* ------------------------------------------------------------------ */

/* The paper uplifts one scene at a time; batching is this library's form
 * for workloads of many scenes with uneven sizes.  Each item is the
 * argument set of one scoup_uplift call (same meaning and layout); C, K and
 * accum_mode are common to the batch. */
typedef struct scoup_batch_item {
  scoup_scene scene;
  const scoup_camera* cams;     /* HOST [V]; read when the batch is captured */
  int32_t V;
  const int32_t* region_maps;   /* DEVICE, views packed as for scoup_uplift */
  const int64_t* map_offsets;   /* HOST [V] */
  int32_t R_total;
  const int32_t* code_idx;      /* DEVICE [R_total, s] */
  const float* code_val;        /* DEVICE [R_total, s] */
  int32_t s;
  float* accum;                 /* DEVICE [n, C] ([2, n, C] when compensated) */
  int32_t* topk_idx;            /* DEVICE [n, K] or NULL */
  float* topk_val;              /* DEVICE [n, K] or NULL */
} scoup_batch_item;

typedef struct scoup_plan scoup_plan;  /* opaque */

typedef struct scoup_tune_entry {
  int32_t lanes;
  int32_t warp_w;
  float ms;             /* best of two timed runs on the view sample */
  int32_t chunk_views;  /* 0: scenes on lanes; > 0: the chunked form (scoup_plan_set_chunk) */
} scoup_tune_entry;

#define SCOUP_MAX_TUNE 24
#define SCOUP_MAX_CHUNK_VIEWS 64
typedef struct scoup_plan_info {
  int32_t lanes;            /* scenes run concurrently on this many streams */
  int32_t warp_w;           /* tile-kernel warp pixel block: warp_w x (32 / warp_w) */
  int32_t tuned;            /* 1 once scoup_autotune has chosen lanes and warp_w */
  int32_t graph_kernels;    /* kernel launches in one replay of the captured graph (0 before) */
  int64_t workspace_bytes;  /* device memory held by the lane workspaces and the chunked form */
  int32_t n_tune;
  scoup_tune_entry tune[SCOUP_MAX_TUNE];  /* the autotuner's measurements */
  int32_t chunk_views;      /* 0: scenes on lanes; > 0: views per chunk of the chunked form */
} scoup_plan_info;

#define SCOUP_BATCH_EAGER 1  /* scoup_uplift_batched flag: launch directly, no graph */

/* Creates a plan for the batch: counts every view's (Gaussian, tile) pairs
 * exactly (synchronising `stream`), sizes one uplift workspace for the
 * largest scene and allocates it for each lane (default lanes: min(4, B),
 * warp block 8x4).  The plan keeps a copy of `items` (the arrays they point
 * to must stay valid and unchanged in size while the plan lives).  The plan
 * owns its device memory until scoup_plan_destroy. */
int scoup_plan_create(const scoup_batch_item* items, int32_t B, int32_t C, int32_t K, int32_t accum_mode,
                      scoup_plan** plan, void* stream);

/* Sets the lane count (1..8) and the tile-kernel warp block width (4, 8 or
 * 16) by hand; drops a captured graph. */
int scoup_plan_set(scoup_plan* plan, int32_t lanes, int32_t warp_w);

/* Selects the batch's execution form.  chunk_views = 0 (the default): each
 * lane runs whole scenes one after another, every view with its own
 * projection, binning and tile launch.  chunk_views in [1, 64]: the views of
 * all scenes are interleaved (view r of every scene, then view r + 1, ...)
 * and cut into chunks of chunk_views views; each view of a chunk is projected
 * and binned into a view workspace of its own, then ONE persistent tile launch
 * composites every (scene, view, tile) item of the chunk, its CTAs taking
 * items from an atomic counter; `lanes` chunks are in flight on the lanes'
 * streams.  Results are those of scoup_uplift per item (the order of FP32
 * sums aside).  The chunked form's device memory (every scene's sorted copy
 * and lanes x chunk_views view workspaces) is allocated at the next run, which
 * then synchronises the device once.  Drops a captured graph. */
int scoup_plan_set_chunk(scoup_plan* plan, int32_t chunk_views);

/* Autotuner: runs the batch restricted to `sample_views` evenly spaced views
 * per scene for every lanes in {1, 2, 4, 8} (<= B) and warp block in
 * {8x4, 16x2, 4x8}, then the chunked form (chunk_views 4, 8 and 16 on 1, 2
 * or 4 lanes (<= B), with the best warp block), times each (CUDA events on `stream`,
 * best of two after a warm-up) and keeps the fastest (scoup_plan_info_get
 * lists the timings).
 * Overwrites the items' accum and Top-K outputs; refused with
 * SCOUP_ACCUM_CONTINUE.  Synchronises `stream`. */
int scoup_autotune(scoup_plan* plan, int32_t sample_views, void* stream);

/* Uplifts every scene of the batch (results as scoup_uplift per item).  The
 * first call captures the whole batch -- fork to the lanes, every launch of
 * every scene, a copy of each scene's counters, join -- into a CUDA graph on
 * `stream` (the stream must not be capturing already); later calls replay
 * it with one graph launch.  Camera parameters and map offsets are read
 * when the graph is captured.  With SCOUP_BATCH_EAGER the launches are
 * issued directly (same lanes, no graph).  Asynchronous; do not run the same
 * plan on two streams at once (the lanes' workspaces are shared). */
int scoup_uplift_batched(scoup_plan* plan, int32_t flags, void* stream);

/* Per-scene counters of the last batched run (HOST stats[B]); synchronises
 * `stream` and returns the first device-side error of any scene. */
int scoup_plan_stats(scoup_plan* plan, scoup_stats* stats, void* stream);

int scoup_plan_info_get(const scoup_plan* plan, scoup_plan_info* info);

/* Frees the plan's device memory, streams and graph (NULL is accepted). */
int scoup_plan_destroy(scoup_plan* plan);

/* ------------------------------------------------------------------ */
/* Codebook decode and text similarity (tensor cores, BF16 inputs)      */
/* ------------------------------------------------------------------ */

/* Workspace bytes for scoup_decode with P rows, C atoms of dimension D. */
size_t scoup_decode_workspace_size(int64_t P, int32_t C, int32_t D);

/* Codebook decode of rendered sparse codes into features (Sec. 4.3, Eq. 8):
 *   features[p][d] = sum_c codes[p][c] codebook[c][d]
 * computed on the tensor cores with BF16 operands and FP32 accumulation.
 *  codes       DEVICE [P, C] row-major, float32 (codes_dtype 0; rounded to
 *              bf16 in the workspace) or bf16 (codes_dtype 1), 16-byte aligned.
 *  codebook    DEVICE float32 [C, D] row-major (rounded to bf16).
 *  features    DEVICE [P, D] row-major, float32 (out_dtype 0) or bf16
 *              (out_dtype 1, round to nearest even), 16-byte aligned.
 *  feat_norm2  DEVICE float32 [P] or NULL: with out_dtype 1, receives the
 *              squared norm of each stored (rounded) feature row, the input
 *              scoup_similarity wants; ignored with out_dtype 0.
 *  workspace   DEVICE, >= scoup_decode_workspace_size(P, C, D) bytes.
 * Limits: C a multiple of 8 in [8, 4096]; D a multiple of 16, >= 16.
 * Asynchronous on `stream`; a device-side timeout (a tensor-core pipeline
 * wait that gave up) is reported by scoup_read_stats on the workspace as
 * status SCOUP_ERR_TIMEOUT. */
int scoup_decode(const void* codes, int32_t codes_dtype, int64_t P, int32_t C, const float* codebook,
                 int32_t D, void* features, int32_t out_dtype, float* feat_norm2, void* workspace,
                 size_t ws_bytes, void* stream);

/* Workspace bytes for scoup_similarity with P feature rows of dimension D
 * against Q text vectors. */
size_t scoup_similarity_workspace_size(int64_t P, int32_t D, int32_t Q);

/* Cosine similarity of decoded features to text embeddings (the open-
 * vocabulary query of App. B):
 *   out[p][q] = <f_p, t_q> / (|f_p| |t_q|),  0 where |f_p| < 1e-12 or |t_q| = 0
 * with BF16 operands and FP32 accumulation on the tensor cores.
 *  features    DEVICE bf16 [P, D] row-major, 16-byte aligned (scoup_decode
 *              with out_dtype 1).
 *  feat_norm2  DEVICE float32 [P] squared feature norms (as scoup_decode
 *              writes them), or NULL to compute them here.
 *  text        DEVICE float32 [Q, D] (rounded to bf16; |t_q| is the norm of
 *              the rounded vector).
 *  out         DEVICE float32 [P, Q].
 * Limits: D a multiple of 8; Q a multiple of 16 in [16, 256] (pad the text
 * set with zero rows).  Asynchronous; errors as for scoup_decode. */
int scoup_similarity(const void* features, int64_t P, int32_t D, const float* feat_norm2, const float* text,
                     int32_t Q, float* out, void* workspace, size_t ws_bytes, void* stream);

/* Backward of the decode (Eq. 8) for the differentiable render: with
 * F = What C, dL/dWhat = dL/dF C^T, a [P, D] x [D, C] contraction on the
 * tensor cores (the codebook rows are its K-major operand as stored).
 *  dF         DEVICE [P, D], float32 (dF_dtype 0, rounded to bf16 inside, in
 *             chunks of the workspace) or bf16 (dF_dtype 1), 16-byte aligned.
 *  codebook   DEVICE float32 [C, D] (rounded to bf16 inside).
 *  dcodes     DEVICE float32 [P, C], 16-byte aligned: overwritten.
 *  C          multiple of 16 in [16, 4096]; D a positive multiple of 8.
 *  workspace  DEVICE, >= scoup_decode_backward_workspace_size(P, C, D) bytes.
 * BF16 operands, FP32 accumulation in tensor memory.  Asynchronous.
 * scoup_decode_backward_fp32 is the FP32 SIMT comparison form (float32 dF,
 * no workspace, any P, C, D >= 1). */
size_t scoup_decode_backward_workspace_size(int64_t P, int32_t C, int32_t D);
int scoup_decode_backward(const void* dF, int32_t dF_dtype, int64_t P, int32_t D, const float* codebook, int32_t C,
                          float* dcodes, void* workspace, size_t ws_bytes, void* stream);
int scoup_decode_backward_fp32(const float* dF, int64_t P, int32_t D, const float* codebook, int32_t C,
                               float* dcodes, void* stream);

/* The L2 loss of the differentiable render against per-pixel region targets
 * and its gradient: the target of pixel p is the decoded code of its region,
 * F*(p) = sum_j v_j C[j] over code_{r(p)} (the region codes of Eq. 5 and the
 * codebook of Eq. 8); L = sum over labelled pixels of |F(p) - F*(p)|^2 and
 * dL/dF(p) = 2 (F(p) - F*(p)) (zero at unlabelled pixels, region -1).
 *  F           DEVICE [P, D] float32 (F_dtype 0) or bf16 (F_dtype 1).
 *  region_map  DEVICE int32 [P]: region of each pixel (row of the code table), -1 none.
 *  code_idx, code_val  DEVICE [R, s] (atom -1 = padding); codebook DEVICE float32 [C, D].
 *  dF          DEVICE [P, D] float32 (dF_dtype 0) or bf16 (dF_dtype 1): overwritten.
 *  loss        DEVICE double: L is added to it (FP32 terms, FP64 sum), or NULL.
 *  workspace   DEVICE, >= scoup_region_l2_grad_workspace_size(R, D) bytes
 *              (the decoded region targets, FP32).
 * A region id >= R or an atom >= C sets the device status read by
 * scoup_read_stats(workspace) (SCOUP_ERR_DEVICE_CHECK).  Asynchronous. */
size_t scoup_region_l2_grad_workspace_size(int32_t R, int32_t D);
int scoup_region_l2_grad(const void* F, int32_t F_dtype, int64_t P, int32_t D, const int32_t* region_map,
                         const int32_t* code_idx, const float* code_val, int32_t R, int32_t s,
                         const float* codebook, int32_t C, void* dF, int32_t dF_dtype, double* loss,
                         void* workspace, size_t ws_bytes, void* stream);

/* FP32 comparison forms of scoup_decode and scoup_similarity: the same
 * results computed with FP32 operands and FP32 FFMA accumulation on the SIMT
 * cores (no rounding of the inputs), for measuring the BF16 forms against.
 *  scoup_decode_fp32:     codes float32 [P, C], codebook float32 [C, D],
 *                         features float32 [P, D].  No workspace.
 *  scoup_similarity_fp32: features float32 [P, D], text float32 [Q, D],
 *                         out float32 [P, Q]; workspace as for
 *                         scoup_similarity (scoup_similarity_workspace_size).
 * All DEVICE pointers; asynchronous on `stream`; any P, C, D, Q >= 1. */
int scoup_decode_fp32(const float* codes, int64_t P, int32_t C, const float* codebook, int32_t D,
                      float* features, void* stream);
int scoup_similarity_fp32(const float* features, int64_t P, int32_t D, const float* text, int32_t Q,
                          float* out, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Uplift without a caller-provided workspace                           */
/* ------------------------------------------------------------------ */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: a host application whose memory manager
 * owns every device allocation and hands out no scratch buffers, or a plugin
 * running inside such a host with no allocator to call.
 *
 * Same arguments and results as scoup_uplift, but the scratch space lives in
 * a fixed array inside this library (scoup_uplift_noalloc_max_bytes() bytes,
 * 32 MiB, held on every GPU that loads the library until the process exits).
 * The call allocates nothing: it calls no cudaMalloc/cudaFree or any other
 * allocating routine.  Caller-owned inputs and outputs are as for
 * scoup_uplift (accum, topk_idx, topk_val are still the caller's).
 *  - Scenes whose fixed scratch (projection records, counters; see
 *    scoup_uplift_workspace_size with dup_capacity 0) exceeds the array are
 *    rejected with SCOUP_ERR_INVALID_ARG and a message; per-view tile lists
 *    use what is left, and a view that needs more returns SCOUP_ERR_CAPACITY.
 *  - The call synchronises `stream` and returns the device status; stats
 *    (host, optional) receives the counters.
 *  - The first call on each device looks up the device address of the array
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept per device and driver
 *    context: after a device reset (a new primary context) the next call
 *    looks it up again. 
 *  - Every call on a device shares the one array and leaves its contents
 *    behind (each call clears what must start at zero).  Calls that overlap on
 *    the GPU -- from several host threads or on several streams at once --
 *    race on the array and give wrong results: serialise them. */
size_t scoup_uplift_noalloc_max_bytes(void);
int scoup_uplift_noalloc(const scoup_scene* scene, const scoup_camera* cams, int32_t V,
                         const int32_t* region_maps, const int64_t* map_offsets, int32_t R_total,
                         const int32_t* code_idx, const float* code_val, int32_t s, int32_t C,
                         int32_t K, float* accum, int32_t accum_mode, int32_t* topk_idx,
                         float* topk_val, scoup_stats* stats, void* stream);

/* ------------------------------------------------------------------ */
/* Profiling hooks                                                     */
/* ------------------------------------------------------------------ */

/* Phases timed by the profiling hooks. */
#define SCOUP_PHASE_TAU 0          /* spatial reorder of the scene + per-Gaussian alpha threshold */
#define SCOUP_PHASE_PREPROCESS 1   /* projection of one view */
#define SCOUP_PHASE_BINNING 2      /* tile binning of one view (3 kernels) */
#define SCOUP_PHASE_UPLIFT_TILES 3 /* per-tile sort + composite + scatter of one view */
#define SCOUP_PHASE_TOPK 4         /* Top-K + normalisation */
#define SCOUP_PHASE_CODE_TOPK 5    /* per-code Top-K (s > K) */
#define SCOUP_PHASE_RENDER 6       /* per-tile sparse-code rendering of one view */
#define SCOUP_PHASE_RENDER_BWD 7   /* per-tile backward of the rendering */
#define SCOUP_PHASE_DECODE 8       /* codebook decode GEMM */
#define SCOUP_PHASE_SIMILARITY 9   /* cosine similarity to text vectors */
#define SCOUP_NUM_PHASES 16

/* When enable != 0, each later launch group of a phase is bracketed by CUDA
 * events recorded on its stream (process-wide switch). */
int scoup_profile_enable(int32_t enable);

/* Waits for the recorded events and returns, per phase, the summed elapsed
 * milliseconds ms[phase] and the number of timed launch groups
 * launches[phase] since the previous read (arrays of nphases, host). */
int scoup_profile_read(double* ms, int64_t* launches, int32_t nphases);

/* Total number of CUDA kernels this library has launched in the process. */
int64_t scoup_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* SCOUP_H */
