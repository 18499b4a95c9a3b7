/*
 * scoup_oracle.h -- plain CPU reference for SCOUP sparse code uplift.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path
 * never does.  It shares no code, header or constant table with the CUDA
 * library.
 *
 * What it computes (paper section / equation):
 *   - front-to-back alpha-compositing weights e_i(v,p) of a tile-binned 3DGS
 *     rasterizer (Sec. 3, Eq. 2);
 *   - sparse coefficient uplift  w_i = sum e_i(v,p) W_v(p)   (Sec. 4.2, Eq. 5,
 *     Algorithm 1), Z_i omitted as the paper allows;
 *   - Top-K + L1 normalisation  (Eq. 6);
 *   - sparse coefficient rendering  (Eq. 7);
 *   - codebook decode F = W C  (Eq. 8) and cosine similarity to text vectors;
 *   - the gradient of an L2 feature loss through Eq. 7 and Eq. 8 with respect
 *     to the Top-K values and the opacities (derived from Eq. 2 and Eq. 7).
 *
 * Precision: values are FP64.  Discrete rasterizer decisions (cull, 2D
 * radius, tile rectangle, depth order, the sign of the Gaussian exponent and
 * the alpha >= 1/255 test) are taken on the IEEE binary32 projection,
 * evaluated in a fixed operation order, because the GPU kernel takes them in
 * binary32; the alpha test itself is the exact predicate o*exp(power) < 1/255
 * evaluated in FP64 on that binary32 exponent.  The transmittance stop
 * T(1-alpha) < 1e-4 depends on exp() and cannot be reproduced bit for bit;
 * the oracle reports every stop decision within a relative margin of the
 * threshold as "at risk" together with the contribution at stake.
 */
#ifndef SCOUP_ORACLE_H
#define SCOUP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  float viewmat[12];   /* world -> camera, 3x4 row-major; camera x right, y down, z forward */
  float fx, fy, cx, cy;
  int32_t width, height;
} orc_camera;

typedef struct {
  int64_t visible;        /* Gaussians not culled, summed over views */
  int64_t duplicates;     /* (Gaussian, tile) pairs of the tile rectangles */
  int64_t evaluated;      /* (pixel, Gaussian) pairs examined while the pixel was active */
  int64_t contributions;  /* accepted (pixel, Gaussian) pairs: alpha >= 1/255, before the stop */
  int64_t at_risk;        /* stop decisions within the margin of the 1e-4 threshold */
} orc_counts;

typedef struct {
  int32_t visible;        /* 0 = culled */
  int32_t rect[4];        /* tile x_lo, y_lo, x_hi, y_hi (hi exclusive) */
  float depth;            /* camera-space z, binary32 */
  float mx, my;           /* 2D mean in pixel-index coordinates, binary32 */
  float qa, qb, qc;       /* exponent coefficients: power = qa dx^2 + qb dx dy + qc dy^2 */
  float radius;           /* ceil(3 sqrt(lambda_max)), binary32 */
  double mx64, my64;      /* FP64 2D mean */
  double ca64, cb64, cc64;/* FP64 inverse 2D covariance (a, b, c) of [[a b][b c]] */
} orc_proj;

/* Stop decisions with |T(1-alpha)/1e-4 - 1| below this are reported at risk. */
#define ORC_STOP_MARGIN 1e-2

void orc_project(const float* mean, const float* scale, const float* quat,
                 const orc_camera* cam, orc_proj* out);

/* Binary32 exponent of Gaussian p at integer pixel (x, y). */
float orc_power_f32(const orc_proj* p, int x, int y);

/* Contribution list of one pixel: gids/e/alpha front to back (capacity cap).
 * brute = 1 scans all n Gaussians for the pixel instead of using tile lists.
 * Returns the number of accepted contributions (or -1 if cap is too small). */
int orc_pixel_list(const float* means, const float* scales, const float* quats,
                   const float* opacity, int64_t n, const orc_camera* cam,
                   int x, int y, int brute, int cap,
                   int32_t* gid, double* e, double* alpha, double* T_final);

/* Uplift (Eq. 5, Algorithm 1) over V views.  acc[n*C] (FP64, zeroed inside)
 * receives the raw sums sum e * c (Z_i omitted).  risk[n*C] (optional)
 * receives, per entry, the sum of c * e over at-risk stop decisions.
 * rows (optional, nrows) restricts the scatter to the listed Gaussians:
 * acc/risk are then [nrows*C] in that order and only tiles touched by them
 * are composited.  nthreads <= 0 uses the OpenMP default. */
int orc_uplift(const float* means, const float* scales, const float* quats,
               const float* opacity, int64_t n, const orc_camera* cams, int V,
               const int32_t* region_maps, const int64_t* map_offsets,
               const int32_t* code_idx, const float* code_val, int s, int C, int K,
               const int64_t* rows, int64_t nrows,
               double* acc, double* risk, orc_counts* counts, int nthreads);

/* Top-K + L1 normalisation (Eq. 6) of acc[n*C]: positive entries only,
 * ordered by (value desc, index asc), padded with (-1, 0). */
int orc_topk(const double* acc, int64_t n, int C, int K, int32_t* idx, double* val);

/* Sparse coefficient rendering (Eq. 7) of one view: What[H*W*C] (dense,
 * unnormalised), T_final[H*W], risk[H*W] (optional: 1 where a stop decision
 * was at risk). */
int orc_render(const float* means, const float* scales, const float* quats,
               const float* opacity, int64_t n, const int32_t* topk_idx,
               const double* topk_val, int K, int C, const orc_camera* cam,
               double* What, double* T_final, uint8_t* risk, orc_counts* counts,
               int nthreads);

/* Codebook decode (Eq. 8): F[P*D] = What[P*C] x codebook[C*D]. */
void orc_decode(const double* What, int64_t P, int C, const float* codebook, int D, double* F);

/* Cosine similarity of F[P*D] rows with text[Q*D] rows; 0 where |F| < 1e-12. */
void orc_similarity(const double* F, int64_t P, int D, const float* text, int Q, double* out);

/* Entropy of each Gaussian's coefficient distribution (the entropy analysis
 * of Top-K filtering): with p_l = w_l / sum_l w_l over the positive entries of
 * row i, H_i = -sum_l p_l log p_l; a row with no positive entry gets 0. */
void orc_entropy(const double* acc, int64_t n, int C, double* H);

/* Entropy filter: keep[i] = 1 for the `keep` rows of lowest entropy (ties to
 * the lower index), 0 for the others. */
void orc_entropy_filter(const double* H, int64_t n, int64_t keep, unsigned char* keep_mask);

/* Relevancy score of a query (App. B, Eq. 9): for each pixel p,
 * R(p) = min_k e^{a s_q} / (e^{a s_q} + e^{a s_k}) with s_q the similarity to the
 * query and s_k the similarities to the n_canon canonical phrases, a = alpha. */
void orc_relevancy(const double* s_query, const double* s_canon, int64_t P, int n_canon, double alpha,
                   double* R);

/* Gradient through Eq. 7 of a loss with dL/dWhat given per pixel:
 * d_val[n*K] += sum_p e_i(p) g_p[idx_ik];
 * d_opacity[n] += sum_p dalpha/do * (T_i (g_p . w_i) - S_after / (1 - alpha_i)). */
int orc_render_backward(const float* means, const float* scales, const float* quats,
                        const float* opacity, int64_t n, const int32_t* topk_idx,
                        const double* topk_val, int K, int C, const orc_camera* cam,
                        const double* dL_dWhat, double* d_val, double* d_opacity);

void orc_free(void* p);

#ifdef __cplusplus
}
#endif
#endif
