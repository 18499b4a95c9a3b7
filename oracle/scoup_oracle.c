/*
 * scoup_oracle.c -- plain CPU reference for SCOUP sparse code uplift.
 *
 * TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU
 * baseline leg load this file's library.  Nothing here is shared with the
 * CUDA path.  Every function is a direct restatement of the paper's
 * definitions, with no blocking, fusion or reordering beyond them:
 *
 *   Sec. 3, Eq. 2     e_i = alpha_i prod_{j<i} (1 - alpha_j), alpha_i = o_i G_i^2D,
 *                     over the Gaussians of a tile-based rasterizer ordered
 *                     front to back (standard 3DGS projection with the EWA
 *                     2D covariance, 16x16 tiles).
 *   Sec. 4.2, Eq. 5   w_i = sum_{(v,p)} e_i(v,p) W_v(p)  (Z_i omitted, Eq. 6 text)
 *   Algorithm 1       loop order views -> pixels -> Gaussians -> code entries
 *   Eq. 6             Top_K(w_i) / |Top_K(w_i)|_1, only where w_i != 0
 *   Eq. 7             What_v(p) = sum_i w^_i e_i(v,p)
 *   Eq. 8             F_v(p) = What_v(p) C
 *
 * The paper cites the standard rasterizer without constants; the oracle uses
 * the standard 3DGS ones: near plane 0.2, 0.3 px^2 low-pass dilation, 1.3x
 * frustum clamp of the Jacobian, radius ceil(3 sqrt(lambda_max)) with a 0.1
 * eigenvalue floor, alpha capped at 0.99, alpha < 1/255 skipped, stop before a
 * Gaussian that would bring T(1-alpha) below 1e-4, pixel (x, y) sampled at the
 * image point (x + 0.5, y + 0.5), depth ties broken by Gaussian index.
 *
 * Decisions vs values: see scoup_oracle.h.  The binary32 projection below is
 * written in one fixed operation order (compiled with contraction off) so the
 * discrete outcomes equal those of any binary32 evaluation in that order; all
 * contribution values come from the separate FP64 projection.
 */
#include "scoup_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TILE 16

/* ------------------------------------------------------------------------ */
/* Projection, binary32 decision path (fixed evaluation order)               */
/* ------------------------------------------------------------------------ */

static int tile_clamp(float v, int g)
{
  if (!(v > 0.0f)) return 0;
  if (v > (float)g) return g;
  return (int)v;
}

static void project_f32(const float* m, const float* s, const float* q,
                        const orc_camera* cam, orc_proj* o)
{
  const float* W = cam->viewmat;
  o->visible = 0;
  float t0 = W[0] * m[0] + W[1] * m[1] + W[2] * m[2] + W[3];
  float t1 = W[4] * m[0] + W[5] * m[1] + W[6] * m[2] + W[7];
  float t2 = W[8] * m[0] + W[9] * m[1] + W[10] * m[2] + W[11];
  o->depth = t2;
  if (!(t2 > 0.2f)) return;                                  /* near plane */

  /* rotation of the normalised quaternion (w, x, y, z) */
  float qn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  float inv = 1.0f / sqrtf(qn);
  float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
  float R[3][3];
  R[0][0] = 1.0f - 2.0f * (y * y + z * z);
  R[0][1] = 2.0f * (x * y - w * z);
  R[0][2] = 2.0f * (x * z + w * y);
  R[1][0] = 2.0f * (x * y + w * z);
  R[1][1] = 1.0f - 2.0f * (x * x + z * z);
  R[1][2] = 2.0f * (y * z - w * x);
  R[2][0] = 2.0f * (x * z - w * y);
  R[2][1] = 2.0f * (y * z + w * x);
  R[2][2] = 1.0f - 2.0f * (x * x + y * y);

  /* Sigma3 = (R S)(R S)^T */
  float M[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
  float S3[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      S3[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];

  /* EWA: J (with 1.3x frustum clamp of the tangent), T = J Rv, Sigma2 = T Sigma3 T^T */
  float limx = 1.3f * (0.5f * (float)cam->width / cam->fx);
  float limy = 1.3f * (0.5f * (float)cam->height / cam->fy);
  float txz = t0 / t2, tyz = t1 / t2;
  float txc = fminf(limx, fmaxf(-limx, txz)) * t2;
  float tyc = fminf(limy, fmaxf(-limy, tyz)) * t2;
  float tz2 = t2 * t2;
  float j00 = cam->fx / t2;
  float j02 = -(cam->fx * txc) / tz2;
  float j11 = cam->fy / t2;
  float j12 = -(cam->fy * tyc) / tz2;
  float T[2][3];
  for (int k = 0; k < 3; ++k) {
    T[0][k] = j00 * W[k] + j02 * W[8 + k];
    T[1][k] = j11 * W[4 + k] + j12 * W[8 + k];
  }
  float U[2][3];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k)
      U[a][k] = T[a][0] * S3[0][k] + T[a][1] * S3[1][k] + T[a][2] * S3[2][k];
  float ca2 = U[0][0] * T[0][0] + U[0][1] * T[0][1] + U[0][2] * T[0][2] + 0.3f;
  float cb2 = U[0][0] * T[1][0] + U[0][1] * T[1][1] + U[0][2] * T[1][2];
  float cc2 = U[1][0] * T[1][0] + U[1][1] * T[1][1] + U[1][2] * T[1][2] + 0.3f;

  float det = ca2 * cc2 - cb2 * cb2;
  if (!(det > 0.0f)) return;
  float idet = 1.0f / det;
  float con_a = cc2 * idet, con_b = -cb2 * idet, con_c = ca2 * idet;

  float mid = 0.5f * (ca2 + cc2);
  float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
  float r = ceilf(3.0f * sqrtf(lam));

  float mx = cam->fx * txz + cam->cx - 0.5f;
  float my = cam->fy * tyz + cam->cy - 0.5f;

  int gx = (cam->width + TILE - 1) / TILE, gy = (cam->height + TILE - 1) / TILE;
  int xlo = tile_clamp(floorf((mx - r) / 16.0f), gx);
  int xhi = tile_clamp(floorf((mx + r + 15.0f) / 16.0f), gx);
  int ylo = tile_clamp(floorf((my - r) / 16.0f), gy);
  int yhi = tile_clamp(floorf((my + r + 15.0f) / 16.0f), gy);
  if (xhi <= xlo || yhi <= ylo) return;                      /* touches no tile */

  o->visible = 1;
  o->rect[0] = xlo; o->rect[1] = ylo; o->rect[2] = xhi; o->rect[3] = yhi;
  o->mx = mx; o->my = my;
  o->qa = -0.5f * con_a;
  o->qb = -con_b;
  o->qc = -0.5f * con_c;
  o->radius = r;
}

/* power = qa dx^2 + qb dx dy + qc dy^2, evaluated as dx*(qa*dx + qb*dy) + (qc*dy)*dy
 * with the inner and outer sums fused (two fmaf) and the products rounded. */
float orc_power_f32(const orc_proj* p, int x, int y)
{
  float dx = p->mx - (float)x;
  float dy = p->my - (float)y;
  float qbdy = p->qb * dy;
  float qcdy = p->qc * dy;
  float qcdy2 = qcdy * dy;
  return fmaf(dx, fmaf(p->qa, dx, qbdy), qcdy2);
}

/* ------------------------------------------------------------------------ */
/* Projection, FP64 value path (textbook matrix form)                        */
/* ------------------------------------------------------------------------ */

static void project_f64(const float* mf, const float* sf, const float* qf,
                        const orc_camera* cam, orc_proj* o)
{
  double W[3][3], tv[3], m[3], s[3], q[4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) W[i][j] = cam->viewmat[4 * i + j];
    tv[i] = cam->viewmat[4 * i + 3];
    m[i] = mf[i];
    s[i] = sf[i];
  }
  double qnorm = 0.0;
  for (int i = 0; i < 4; ++i) { q[i] = qf[i]; qnorm += q[i] * q[i]; }
  qnorm = sqrt(qnorm);
  for (int i = 0; i < 4; ++i) q[i] /= qnorm;

  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = W[i][0] * m[0] + W[i][1] * m[1] + W[i][2] * m[2] + tv[i];

  double w = q[0], x = q[1], y = q[2], z = q[3];
  double R[3][3] = {
    {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
    {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
    {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  /* Sigma3 = R diag(s^2) R^T */
  double S3[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += R[i][k] * s[k] * s[k] * R[j][k];
      S3[i][j] = acc;
    }
  double limx = 1.3 * cam->width / (2.0 * cam->fx);
  double limy = 1.3 * cam->height / (2.0 * cam->fy);
  double tx = fmin(limx, fmax(-limx, t[0] / t[2])) * t[2];
  double ty = fmin(limy, fmax(-limy, t[1] / t[2])) * t[2];
  double J[2][3] = {{cam->fx / t[2], 0.0, -cam->fx * tx / (t[2] * t[2])},
                    {0.0, cam->fy / t[2], -cam->fy * ty / (t[2] * t[2])}};
  /* JW = J W ; Sigma2 = JW Sigma3 JW^T */
  double JW[2][3];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) JW[a][k] = J[a][0] * W[0][k] + J[a][1] * W[1][k] + J[a][2] * W[2][k];
  double S2[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double acc = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += JW[a][i] * S3[i][j] * JW[b][j];
      S2[a][b] = acc;
    }
  double a = S2[0][0] + 0.3, b = S2[0][1], c = S2[1][1] + 0.3;
  double det = a * c - b * b;
  o->ca64 = c / det;
  o->cb64 = -b / det;
  o->cc64 = a / det;
  o->mx64 = cam->fx * t[0] / t[2] + cam->cx - 0.5;
  o->my64 = cam->fy * t[1] / t[2] + cam->cy - 0.5;
}

void orc_project(const float* mean, const float* scale, const float* quat,
                 const orc_camera* cam, orc_proj* out)
{
  memset(out, 0, sizeof(*out));
  project_f32(mean, scale, quat, cam, out);
  if (out->visible) project_f64(mean, scale, quat, cam, out);
}

/* ------------------------------------------------------------------------ */
/* Per-view state: projections and depth-sorted tile lists                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  float depth;
  int32_t gid;
} depth_key;

static int cmp_depth_key(const void* pa, const void* pb)
{
  const depth_key* a = (const depth_key*)pa;
  const depth_key* b = (const depth_key*)pb;
  if (a->depth < b->depth) return -1;
  if (a->depth > b->depth) return 1;
  return (a->gid > b->gid) - (a->gid < b->gid);
}

typedef struct {
  const orc_camera* cam;
  int gx, gy, ntiles;
  int64_t n;
  const float* opacity;
  orc_proj* P;
  int64_t* tile_start;  /* [ntiles + 1] */
  int32_t* tile_list;   /* gids, each tile sorted by (depth, gid) */
} view_ctx;

static void view_free(view_ctx* v)
{
  free(v->P);
  free(v->tile_start);
  free(v->tile_list);
  memset(v, 0, sizeof(*v));
}

/* Project every Gaussian for this view and build the depth-sorted candidate
 * lists of the tiles flagged in `want` (all tiles when want == NULL). */
static int view_setup_tiles(view_ctx* v, const float* means, const float* scales,
                            const float* quats, const float* opacity, int64_t n,
                            const orc_camera* cam, orc_counts* cnt,
                            const int64_t* rows, int64_t nrows)
{
  memset(v, 0, sizeof(*v));
  v->cam = cam;
  v->n = n;
  v->opacity = opacity;
  v->gx = (cam->width + TILE - 1) / TILE;
  v->gy = (cam->height + TILE - 1) / TILE;
  v->ntiles = v->gx * v->gy;
  v->P = (orc_proj*)malloc(sizeof(orc_proj) * (size_t)(n > 0 ? n : 1));
  v->tile_start = (int64_t*)calloc((size_t)v->ntiles + 1, sizeof(int64_t));
  uint8_t* want = (uint8_t*)calloc((size_t)v->ntiles, 1);
  if (!v->P || !v->tile_start || !want) { free(want); view_free(v); return -1; }

#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    orc_project(means + 3 * i, scales + 3 * i, quats + 4 * i, cam, &v->P[i]);

  if (rows) {
    for (int64_t r = 0; r < nrows; ++r) {
      const orc_proj* p = &v->P[rows[r]];
      if (!p->visible) continue;
      for (int ty = p->rect[1]; ty < p->rect[3]; ++ty)
        for (int tx = p->rect[0]; tx < p->rect[2]; ++tx) want[ty * v->gx + tx] = 1;
    }
  } else {
    memset(want, 1, (size_t)v->ntiles);
  }

  /* count (Gaussian, tile) pairs per wanted tile */
  int64_t visible = 0, dups = 0;
  for (int64_t i = 0; i < n; ++i) {
    const orc_proj* p = &v->P[i];
    if (!p->visible) continue;
    ++visible;
    dups += (int64_t)(p->rect[2] - p->rect[0]) * (p->rect[3] - p->rect[1]);
    for (int ty = p->rect[1]; ty < p->rect[3]; ++ty)
      for (int tx = p->rect[0]; tx < p->rect[2]; ++tx)
        if (want[ty * v->gx + tx]) v->tile_start[ty * v->gx + tx + 1]++;
  }
  for (int t = 0; t < v->ntiles; ++t) v->tile_start[t + 1] += v->tile_start[t];
  int64_t listed = v->tile_start[v->ntiles];
  v->tile_list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(listed > 0 ? listed : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)v->ntiles);
  if (!v->tile_list || !fill) { free(fill); free(want); view_free(v); return -1; }
  memcpy(fill, v->tile_start, sizeof(int64_t) * (size_t)v->ntiles);
  for (int64_t i = 0; i < n; ++i) {
    const orc_proj* p = &v->P[i];
    if (!p->visible) continue;
    for (int ty = p->rect[1]; ty < p->rect[3]; ++ty)
      for (int tx = p->rect[0]; tx < p->rect[2]; ++tx)
        if (want[ty * v->gx + tx]) v->tile_list[fill[ty * v->gx + tx]++] = (int32_t)i;
  }
  free(fill);
  free(want);

  /* front-to-back order: (depth, gid) ascending */
#pragma omp parallel
  {
    depth_key* buf = NULL;
    size_t cap = 0;
#pragma omp for schedule(dynamic, 4)
    for (int t = 0; t < v->ntiles; ++t) {
      int64_t a = v->tile_start[t], b = v->tile_start[t + 1];
      size_t len = (size_t)(b - a);
      if (len > cap) { free(buf); cap = len; buf = (depth_key*)malloc(sizeof(depth_key) * cap); }
      for (size_t k = 0; k < len; ++k) {
        buf[k].gid = v->tile_list[a + (int64_t)k];
        buf[k].depth = v->P[buf[k].gid].depth;
      }
      qsort(buf, len, sizeof(depth_key), cmp_depth_key);
      for (size_t k = 0; k < len; ++k) v->tile_list[a + (int64_t)k] = buf[k].gid;
    }
    free(buf);
  }
  if (cnt) { cnt->visible += visible; cnt->duplicates += dups; }
  return 0;
}

static int view_setup(view_ctx* v, const float* means, const float* scales,
                      const float* quats, const float* opacity, int64_t n,
                      const orc_camera* cam, orc_counts* cnt)
{
  return view_setup_tiles(v, means, scales, quats, opacity, n, cam, cnt, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* Front-to-back compositing of one pixel (Eq. 2)                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t gid;
  double e;        /* contribution weight alpha * T */
  double alpha;
  double T;        /* transmittance before this Gaussian */
} hit_t;

typedef struct {
  hit_t* hits;  int nh, caph;
  hit_t* risk;  int nr, capr;
  double T_final;
  int64_t evaluated;
} pixel_out;

static int push_hit(hit_t** arr, int* nh, int* cap, hit_t h)
{
  if (*nh == *cap) {
    int nc = *cap ? 2 * *cap : 64;
    hit_t* na = (hit_t*)realloc(*arr, sizeof(hit_t) * (size_t)nc);
    if (!na) return -1;
    *arr = na;
    *cap = nc;
  }
  (*arr)[(*nh)++] = h;
  return 0;
}

/* Composite the candidates `list[0..len)` (front to back) at pixel (x, y).
 * Accepted contributions go to out->hits; stop decisions within
 * ORC_STOP_MARGIN of the threshold, and the contributions a binary32
 * evaluation could add or drop there, go to out->risk. */
static int composite_pixel(const orc_proj* P, const float* opacity,
                           const int32_t* list, int64_t len, int x, int y, pixel_out* out)
{
  const double stop = 1e-4, hi = 1e-4 * (1.0 + ORC_STOP_MARGIN), lo = 1e-4 * (1.0 - ORC_STOP_MARGIN);
  double T = 1.0;
  int stopped = 0;
  out->nh = 0;
  out->nr = 0;
  out->evaluated = 0;
  out->T_final = 1.0;
  for (int64_t k = 0; k < len; ++k) {
    const int32_t g = list[k];
    const orc_proj* p = &P[g];
    if (!stopped) out->evaluated++;
    /* decisions on the binary32 exponent */
    float pw = orc_power_f32(p, x, y);
    if (pw > 0.0f) continue;
    if ((double)opacity[g] * exp((double)pw) < 1.0 / 255.0) continue;
    /* values in FP64 */
    double dx = p->mx64 - (double)x, dy = p->my64 - (double)y;
    double power = -0.5 * (p->ca64 * dx * dx + p->cc64 * dy * dy) - p->cb64 * dx * dy;
    double alpha = fmin(0.99, (double)opacity[g] * exp(power));
    double test = T * (1.0 - alpha);
    hit_t h = {g, alpha * T, alpha, T};
    if (!stopped) {
      if (test < stop) {
        stopped = 1;
        out->T_final = T;
        if (test < lo) break;
        if (push_hit(&out->risk, &out->nr, &out->capr, h)) return -1;
        T = test;          /* continue the hypothetical walk past the stop */
      } else {
        if (push_hit(&out->hits, &out->nh, &out->caph, h)) return -1;
        if (test < hi && push_hit(&out->risk, &out->nr, &out->capr, h)) return -1;
        T = test;
      }
    } else {
      if (test < lo) break;
      if (push_hit(&out->risk, &out->nr, &out->capr, h)) return -1;
      T = test;
    }
  }
  if (!stopped) out->T_final = T;
  return 0;
}

static void pixel_out_free(pixel_out* o)
{
  free(o->hits);
  free(o->risk);
  memset(o, 0, sizeof(*o));
}

/* ------------------------------------------------------------------------ */
/* Single-pixel lists (tile-binned or brute force)                            */
/* ------------------------------------------------------------------------ */

int orc_pixel_list(const float* means, const float* scales, const float* quats,
                   const float* opacity, int64_t n, const orc_camera* cam,
                   int x, int y, int brute, int cap,
                   int32_t* gid, double* e, double* alpha, double* T_final)
{
  pixel_out po;
  memset(&po, 0, sizeof(po));
  int rc = 0;
  if (!brute) {
    view_ctx v;
    if (view_setup(&v, means, scales, quats, opacity, n, cam, NULL)) return -1;
    int t = (y / TILE) * v.gx + (x / TILE);
    rc = composite_pixel(v.P, opacity, v.tile_list + v.tile_start[t],
                         v.tile_start[t + 1] - v.tile_start[t], x, y, &po);
    view_free(&v);
  } else {
    /* every Gaussian, projected on its own; keep those whose rectangle holds
       the pixel's tile; sort by (depth, gid) */
    orc_proj* P = (orc_proj*)malloc(sizeof(orc_proj) * (size_t)(n > 0 ? n : 1));
    depth_key* keys = (depth_key*)malloc(sizeof(depth_key) * (size_t)(n > 0 ? n : 1));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!P || !keys || !list) { free(P); free(keys); free(list); return -1; }
    int tx = x / TILE, ty = y / TILE;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
      orc_project(means + 3 * i, scales + 3 * i, quats + 4 * i, cam, &P[i]);
      if (P[i].visible && tx >= P[i].rect[0] && tx < P[i].rect[2] && ty >= P[i].rect[1] &&
          ty < P[i].rect[3]) {
        keys[m].depth = P[i].depth;
        keys[m].gid = (int32_t)i;
        ++m;
      }
    }
    qsort(keys, (size_t)m, sizeof(depth_key), cmp_depth_key);
    for (int64_t k = 0; k < m; ++k) list[k] = keys[k].gid;
    rc = composite_pixel(P, opacity, list, m, x, y, &po);
    free(P);
    free(keys);
    free(list);
  }
  if (rc) { pixel_out_free(&po); return -1; }
  if (po.nh > cap) { pixel_out_free(&po); return -1; }
  for (int k = 0; k < po.nh; ++k) {
    gid[k] = po.hits[k].gid;
    e[k] = po.hits[k].e;
    alpha[k] = po.hits[k].alpha;
  }
  if (T_final) *T_final = po.T_final;
  int nh = po.nh;
  pixel_out_free(&po);
  return nh;
}

/* ------------------------------------------------------------------------ */
/* Uplift (Eq. 5, Algorithm 1)                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t pix;
  int32_t gid;
  double e;
} rec_t;

typedef struct {
  rec_t* r;
  int64_t n, cap;
} rec_buf;

static int rec_push(rec_buf* b, int32_t pix, int32_t gid, double e)
{
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 256;
    rec_t* na = (rec_t*)realloc(b->r, sizeof(rec_t) * (size_t)nc);
    if (!na) return -1;
    b->r = na;
    b->cap = nc;
  }
  b->r[b->n].pix = pix;
  b->r[b->n].gid = gid;
  b->r[b->n].e = e;
  b->n++;
  return 0;
}

/* Alg. 1 uses TopK(W_v(p)) per pixel; a code with more than K entries keeps
 * its K largest (ties to the lower atom index). */
static void code_keep_mask(const int32_t* idx, const float* val, int s, int K, uint8_t* keep)
{
  for (int a = 0; a < s; ++a) keep[a] = idx[a] >= 0;
  if (s <= K) return;
  for (int a = 0; a < s; ++a) {
    if (!keep[a]) continue;
    int better = 0;
    for (int b = 0; b < s; ++b) {
      if (b == a || idx[b] < 0) continue;
      if (val[b] > val[a] || (val[b] == val[a] && idx[b] < idx[a])) ++better;
    }
    keep[a] = better < K;
  }
}

int orc_uplift(const float* means, const float* scales, const float* quats,
               const float* opacity, int64_t n, const orc_camera* cams, int V,
               const int32_t* region_maps, const int64_t* map_offsets,
               const int32_t* code_idx, const float* code_val, int s, int C, int K,
               const int64_t* rows, int64_t nrows,
               double* acc, double* risk, orc_counts* counts, int nthreads)
{
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const int64_t nout = rows ? nrows : n;
  memset(acc, 0, sizeof(double) * (size_t)nout * (size_t)C);
  if (risk) memset(risk, 0, sizeof(double) * (size_t)nout * (size_t)C);
  if (counts) memset(counts, 0, sizeof(*counts));

  int64_t* row_of = NULL;
  if (rows) {
    row_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!row_of) return -1;
    for (int64_t i = 0; i < n; ++i) row_of[i] = -1;
    for (int64_t r = 0; r < nrows; ++r) row_of[rows[r]] = r;
  }
  uint8_t keep[1024];
  if (s > 1024) { free(row_of); return -1; }

  for (int v = 0; v < V; ++v) {
    const orc_camera* cam = &cams[v];
    const int32_t* rmap = region_maps + map_offsets[v];
    view_ctx vc;
    if (view_setup_tiles(&vc, means, scales, quats, opacity, n, cam, counts, rows, nrows)) {
      free(row_of);
      return -1;
    }

    /* tiles to composite: all, or those touched by the requested rows */
    uint8_t* want = (uint8_t*)calloc((size_t)vc.ntiles, 1);
    rec_buf* hits = (rec_buf*)calloc((size_t)vc.ntiles, sizeof(rec_buf));
    rec_buf* risks = (rec_buf*)calloc((size_t)vc.ntiles, sizeof(rec_buf));
    int64_t* t_eval = (int64_t*)calloc((size_t)vc.ntiles, sizeof(int64_t));
    int64_t* t_risk = (int64_t*)calloc((size_t)vc.ntiles, sizeof(int64_t));
    if (!want || !hits || !risks || !t_eval || !t_risk) { free(row_of); view_free(&vc); return -1; }
    if (rows) {
      for (int64_t r = 0; r < nrows; ++r) {
        const orc_proj* p = &vc.P[rows[r]];
        if (!p->visible) continue;
        for (int ty = p->rect[1]; ty < p->rect[3]; ++ty)
          for (int tx = p->rect[0]; tx < p->rect[2]; ++tx) want[ty * vc.gx + tx] = 1;
      }
    } else {
      memset(want, 1, (size_t)vc.ntiles);
    }

    int failed = 0;
#pragma omp parallel
    {
      pixel_out po;
      memset(&po, 0, sizeof(po));
#pragma omp for schedule(dynamic, 1)
      for (int t = 0; t < vc.ntiles; ++t) {
        if (!want[t]) continue;
        int tx = t % vc.gx, ty = t / vc.gx;
        const int32_t* list = vc.tile_list + vc.tile_start[t];
        int64_t len = vc.tile_start[t + 1] - vc.tile_start[t];
        for (int y = ty * TILE; y < ty * TILE + TILE && y < cam->height; ++y)
          for (int x = tx * TILE; x < tx * TILE + TILE && x < cam->width; ++x) {
            if (composite_pixel(vc.P, opacity, list, len, x, y, &po)) { failed = 1; continue; }
            int32_t pix = y * cam->width + x;
            t_eval[t] += po.evaluated;
            for (int k = 0; k < po.nh; ++k)
              if (rec_push(&hits[t], pix, po.hits[k].gid, po.hits[k].e)) failed = 1;
            if (po.nr) t_risk[t] += 1;
            for (int k = 0; k < po.nr; ++k)
              if (rec_push(&risks[t], pix, po.risk[k].gid, po.risk[k].e)) failed = 1;
          }
      }
      pixel_out_free(&po);
    }

    /* scatter in tile order, pixels row-major within a tile, list order:
       w_i[j] += c_j * e_i(v, p) for every code entry (j, c_j) of the pixel */
    for (int t = 0; t < vc.ntiles && !failed; ++t) {
      for (int pass = 0; pass < 2; ++pass) {
        rec_buf* b = pass == 0 ? &hits[t] : &risks[t];
        double* dst = pass == 0 ? acc : risk;
        if (!dst) continue;
        for (int64_t k = 0; k < b->n; ++k) {
          const rec_t* rc = &b->r[k];
          int64_t row = rows ? row_of[rc->gid] : rc->gid;
          if (row < 0) continue;
          int32_t region = rmap[rc->pix];
          if (region < 0) continue;
          const int32_t* ci = code_idx + (int64_t)region * s;
          const float* cv = code_val + (int64_t)region * s;
          code_keep_mask(ci, cv, s, K, keep);
          for (int a = 0; a < s; ++a)
            if (keep[a]) dst[row * C + ci[a]] += (double)cv[a] * rc->e;
        }
      }
      if (counts) {
        counts->evaluated += t_eval[t];
        counts->contributions += hits[t].n;
        counts->at_risk += t_risk[t];
      }
    }
    for (int t = 0; t < vc.ntiles; ++t) { free(hits[t].r); free(risks[t].r); }
    free(hits); free(risks); free(want); free(t_eval); free(t_risk);
    view_free(&vc);
    if (failed) { free(row_of); return -1; }
  }
  free(row_of);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Top-K + L1 normalisation (Eq. 6)                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  double v;
  int32_t j;
} vj_t;

static int cmp_vj(const void* pa, const void* pb)
{
  const vj_t* a = (const vj_t*)pa;
  const vj_t* b = (const vj_t*)pb;
  if (a->v > b->v) return -1;
  if (a->v < b->v) return 1;
  return (a->j > b->j) - (a->j < b->j);
}

int orc_topk(const double* acc, int64_t n, int C, int K, int32_t* idx, double* val)
{
  vj_t* buf = (vj_t*)malloc(sizeof(vj_t) * (size_t)(C > 0 ? C : 1));
  if (!buf) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int m = 0;
    for (int j = 0; j < C; ++j)
      if (acc[i * C + j] > 0.0) { buf[m].v = acc[i * C + j]; buf[m].j = j; ++m; }
    qsort(buf, (size_t)m, sizeof(vj_t), cmp_vj);
    int take = m < K ? m : K;
    double sum = 0.0;
    for (int k = 0; k < take; ++k) sum += buf[k].v;
    for (int k = 0; k < K; ++k) {
      idx[i * K + k] = k < take ? buf[k].j : -1;
      val[i * K + k] = k < take ? buf[k].v / sum : 0.0;
    }
  }
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sparse coefficient rendering (Eq. 7)                                      */
/* ------------------------------------------------------------------------ */

int orc_render(const float* means, const float* scales, const float* quats,
               const float* opacity, int64_t n, const int32_t* topk_idx,
               const double* topk_val, int K, int C, const orc_camera* cam,
               double* What, double* T_final, uint8_t* risk, orc_counts* counts,
               int nthreads)
{
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  view_ctx vc;
  if (counts) memset(counts, 0, sizeof(*counts));
  if (view_setup(&vc, means, scales, quats, opacity, n, cam, counts)) return -1;
  const int64_t npx = (int64_t)cam->width * cam->height;
  memset(What, 0, sizeof(double) * (size_t)npx * (size_t)C);
  int failed = 0;
  int64_t evaluated = 0, contributions = 0, at_risk = 0;
#pragma omp parallel reduction(+ : evaluated, contributions, at_risk)
  {
    pixel_out po;
    memset(&po, 0, sizeof(po));
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < vc.ntiles; ++t) {
      int tx = t % vc.gx, ty = t / vc.gx;
      const int32_t* list = vc.tile_list + vc.tile_start[t];
      int64_t len = vc.tile_start[t + 1] - vc.tile_start[t];
      for (int y = ty * TILE; y < ty * TILE + TILE && y < cam->height; ++y)
        for (int x = tx * TILE; x < tx * TILE + TILE && x < cam->width; ++x) {
          if (composite_pixel(vc.P, opacity, list, len, x, y, &po)) { failed = 1; continue; }
          int64_t pix = (int64_t)y * cam->width + x;
          double* out = What + pix * C;
          for (int k = 0; k < po.nh; ++k) {
            const int32_t g = po.hits[k].gid;
            for (int a = 0; a < K; ++a) {
              int32_t j = topk_idx[(int64_t)g * K + a];
              if (j >= 0) out[j] += topk_val[(int64_t)g * K + a] * po.hits[k].e;
            }
          }
          if (T_final) T_final[pix] = po.T_final;
          if (risk) risk[pix] = po.nr > 0;
          evaluated += po.evaluated;
          contributions += po.nh;
          at_risk += po.nr > 0;
        }
    }
    pixel_out_free(&po);
  }
  if (counts) {
    counts->evaluated += evaluated;
    counts->contributions += contributions;
    counts->at_risk += at_risk;
  }
  view_free(&vc);
  return failed ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Decode (Eq. 8) and cosine similarity                                      */
/* ------------------------------------------------------------------------ */

void orc_decode(const double* What, int64_t P, int C, const float* codebook, int D, double* F)
{
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < P; ++p)
    for (int d = 0; d < D; ++d) {
      double acc = 0.0;
      for (int c = 0; c < C; ++c) acc += What[p * C + c] * (double)codebook[(int64_t)c * D + d];
      F[p * D + d] = acc;
    }
}

void orc_similarity(const double* F, int64_t P, int D, const float* text, int Q, double* out)
{
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < P; ++p) {
    double nf = 0.0;
    for (int d = 0; d < D; ++d) nf += F[p * D + d] * F[p * D + d];
    nf = sqrt(nf);
    for (int q = 0; q < Q; ++q) {
      double dot = 0.0, nt = 0.0;
      for (int d = 0; d < D; ++d) {
        dot += F[p * D + d] * (double)text[(int64_t)q * D + d];
        nt += (double)text[(int64_t)q * D + d] * (double)text[(int64_t)q * D + d];
      }
      nt = sqrt(nt);
      out[p * Q + q] = (nf < 1e-12 || nt == 0.0) ? 0.0 : dot / (nf * nt);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Backward of Eq. 7 w.r.t. Top-K values and opacities                       */
/* ------------------------------------------------------------------------ */

int orc_render_backward(const float* means, const float* scales, const float* quats,
                        const float* opacity, int64_t n, const int32_t* topk_idx,
                        const double* topk_val, int K, int C, const orc_camera* cam,
                        const double* dL_dWhat, double* d_val, double* d_opacity)
{
  view_ctx vc;
  if (view_setup(&vc, means, scales, quats, opacity, n, cam, NULL)) return -1;
  pixel_out po;
  memset(&po, 0, sizeof(po));
  double* gw = NULL;
  int capg = 0;
  int failed = 0;
  for (int t = 0; t < vc.ntiles && !failed; ++t) {
    int tx = t % vc.gx, ty = t / vc.gx;
    const int32_t* list = vc.tile_list + vc.tile_start[t];
    int64_t len = vc.tile_start[t + 1] - vc.tile_start[t];
    for (int y = ty * TILE; y < ty * TILE + TILE && y < cam->height; ++y)
      for (int x = tx * TILE; x < tx * TILE + TILE && x < cam->width; ++x) {
        if (composite_pixel(vc.P, opacity, list, len, x, y, &po)) { failed = 1; break; }
        const double* g = dL_dWhat + ((int64_t)y * cam->width + x) * C;
        if (po.nh > capg) {
          capg = po.nh;
          double* ng = (double*)realloc(gw, sizeof(double) * (size_t)capg);
          if (!ng) { failed = 1; break; }
          gw = ng;
        }
        /* g . w^_i for every contributor; dL/dval = e * g[idx] */
        for (int k = 0; k < po.nh; ++k) {
          const int32_t i = po.hits[k].gid;
          double dot = 0.0;
          for (int a = 0; a < K; ++a) {
            int32_t j = topk_idx[(int64_t)i * K + a];
            if (j < 0) continue;
            dot += topk_val[(int64_t)i * K + a] * g[j];
            d_val[(int64_t)i * K + a] += po.hits[k].e * g[j];
          }
          gw[k] = dot;
        }
        /* dWhat/dalpha_k = T_k w^_k - sum_{l>k} e_l w^_l / (1 - alpha_k) */
        double S_after = 0.0;
        for (int k = po.nh - 1; k >= 0; --k) {
          const int32_t i = po.hits[k].gid;
          const orc_proj* p = &vc.P[i];
          double dx = p->mx64 - (double)x, dy = p->my64 - (double)y;
          double G = exp(-0.5 * (p->ca64 * dx * dx + p->cc64 * dy * dy) - p->cb64 * dx * dy);
          double dalpha_do = ((double)opacity[i] * G < 0.99) ? G : 0.0;
          double dL_dalpha = po.hits[k].T * gw[k] - S_after / (1.0 - po.hits[k].alpha);
          d_opacity[i] += dalpha_do * dL_dalpha;
          S_after += po.hits[k].e * gw[k];
        }
      }
  }
  free(gw);
  pixel_out_free(&po);
  view_free(&vc);
  return failed ? -1 : 0;
}

void orc_free(void* p) { free(p); }

/* ---- entropy of the coefficient distribution, entropy filter ---------- */

void orc_entropy(const double* acc, int64_t n, int C, double* H)
{
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double* w = acc + i * C;
    double total = 0.0;
    for (int l = 0; l < C; ++l)
      if (w[l] > 0.0) total += w[l];
    double h = 0.0;
    if (total > 0.0)
      for (int l = 0; l < C; ++l)
        if (w[l] > 0.0) {
          const double pl = w[l] / total;
          h -= pl * log(pl);
        }
    H[i] = h;
  }
}

static const double* g_filter_H;

static int cmp_entropy_rank(const void* pa, const void* pb)
{
  const int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
  if (g_filter_H[a] < g_filter_H[b]) return -1;
  if (g_filter_H[a] > g_filter_H[b]) return 1;
  return (a > b) - (a < b);
}

void orc_entropy_filter(const double* H, int64_t n, int64_t keep, unsigned char* keep_mask)
{
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) order[i] = i;
  g_filter_H = H;
  qsort(order, (size_t)n, sizeof(int64_t), cmp_entropy_rank);
  for (int64_t i = 0; i < n; ++i) keep_mask[i] = 0;
  for (int64_t r = 0; r < keep && r < n; ++r) keep_mask[order[r]] = 1;
  free(order);
}

/* ---- relevancy score (App. B) ------------------------------------------ */

void orc_relevancy(const double* s_query, const double* s_canon, int64_t P, int n_canon, double alpha,
                   double* R)
{
  for (int64_t p = 0; p < P; ++p) {
    const double eq = exp(alpha * s_query[p]);
    double r = 1.0;
    for (int k = 0; k < n_canon; ++k) {
      const double ek = exp(alpha * s_canon[p * n_canon + k]);
      const double v = eq / (eq + ek);
      if (v < r) r = v;
    }
    R[p] = r;
  }
}
