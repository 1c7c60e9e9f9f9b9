/*
 * FlashSplat FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct restatement of what the GPU path computes,
 * written from the paper (FlashSplat, arXiv 2409.08270):
 *
 *   Sec. 3.1, Eq. 1   front-to-back alpha blending  X = sum_i x_i alpha_i T_i,
 *                     T_i = prod_{j<i} (1 - alpha_j), Gaussians taken in depth
 *                     order, alpha_i = o_i * (2D Gaussian value at the pixel).
 *   Sec. 3.2, Eq. 6   A_n^i = sum_{v,j,k} alpha_i T_i * [M^v_jk == n].
 *   Sec. 3.3, Eq. 7   the same table with one column per label e = 0..E-1.
 *   Sec. 4.2 / Supp. Sec. 6   the table is filled by walking every mask pixel
 *                     with the rasteriser's alpha compositing, adding
 *                     alpha_i*T_i into the column of the pixel's label.
 *   Sec. 3.4          novel-view masks: each object's Gaussians rendered
 *                     alone, accumulated alpha quantised at tau, the nearest
 *                     passing object chosen by depth (fso_render_masks).
 *   Sec. 4.2          optionally the standard rasteriser's 3-sigma tile
 *                     coverage instead of the exact one (coverage = 1).
 *
 * Everything is double precision.  Conventions the paper leaves open are fixed
 * here and listed, with the reasons, in the repository's design notes:
 *   - 3D covariance  Sigma = R(q) diag(s^2) R(q)^T, q = (w,x,y,z) normalised.
 *   - EWA projection with a 0.3 px^2 low-pass on the 2D covariance diagonal;
 *     the Jacobian is evaluated with tx/tz, ty/tz clamped to 1.3*tan(half-FoV).
 *   - Cull: tz <= 0.2, det(Sigma2D) <= 0, o < 1/255.
 *   - Pixel (u,v) is sampled at (u+0.5, v+0.5); mean2D = (fx tx/tz + cx, ...).
 *   - alpha = min(0.99, o * exp(-0.5 d^T Sigma2D^-1 d)); a Gaussian with
 *     alpha < 1/255 is skipped; if T*(1-alpha) < 1e-4 the pixel stops before
 *     adding that Gaussian.
 *   - Depth order: view-space tz of the mean, ties by lower Gaussian index.
 *
 * The candidate set of a pixel is found through a spatial index (8x8 pixel
 * bins holding every Gaussian whose exact alpha >= 1/255 ellipse bound, plus a
 * one-pixel margin, touches the bin).  With cull_mode = 1 every pixel instead
 * walks every projected Gaussian; both must give the same table, which the
 * tests check.
 *
 * This file shares no code with the CUDA path and must only be called from
 * tests, the smoke check and the CPU-baseline leg of the benchmark.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FSO_ALPHA_MIN (1.0 / 255.0)
#define FSO_ALPHA_MAX 0.99
#define FSO_T_MIN 1e-4
#define FSO_NEAR_PLANE 0.2
#define FSO_LOWPASS 0.3
#define FSO_BIN 8
#define FSO_TILE 16          /* the rasteriser's tile side (Sec. 3.1) */
#define FSO_COVERAGE_3SIGMA 1
#define FSO_CELL 32 /* coarse grid of the tracked-row mode */
#define FSO_HALF_LOG2E 0.72134752044448170368 /* 0.5 log2(e) */

/* Near-threshold model.  An implementation in another precision computes
 * alpha with some relative error; event_rel is the bound assumed for it
 * (default FSO_EVENT_REL: an FP32 rasteriser's alpha is good to a few 1e-6
 * relative near the 1/255 cut, the exponent being a sum of squares of O(1)
 * terms).  A decision is marginal -- it may legitimately go the other way --
 * when it lies within what that error can move:
 *   alpha vs 1/255:      |alpha - 1/255| <= event_rel * 1/255;
 *   T(1 - alpha) vs 1e-4: within event_rel * (1 + sum alpha/(1 - alpha)) of
 *        1e-4 (the relative error alpha's errors carry into the product T
 *        after the pixel's earlier factors and this one), plus 2^-23 per
 *        factor (the product's own rounding), plus the uncertainty of T left
 *        by earlier marginal alpha decisions (`down`).
 * The window only shapes the risk bookkeeping, never the table itself. */
#define FSO_EVENT_REL 1e-5
/* Depths are view-space z in double precision; two Gaussians whose depths
 * agree to 1e-12 relative may be ordered either way by an implementation that
 * computes z with other rounding. */
#define FSO_DEPTH_TIE_REL 1e-12

/* The compositing rule's thresholds (Sec. 3.1 Eq. 1 with the rasteriser's
 * conventions) and the near-threshold window.  Tests move the thresholds
 * within the window to check that the risk bound covers the change. */
typedef struct {
  double alpha_min; /* 1/255: smaller alpha is skipped */
  double t_min;     /* 1e-4: the pixel stops before T would fall below it */
  double ev_rel;    /* relative precision assumed for alpha (see above) */
} fso_rule;

/* flag bits per Gaussian */
#define FSO_FLAG_ALPHA_EDGE 1u   /* alpha within its window of 1/255 */
#define FSO_FLAG_T_EDGE 2u       /* T(1-alpha) within its window of 1e-4 */
#define FSO_FLAG_DEPTH_TIE 4u    /* depth within 1e-12 rel. of a neighbour */
#define FSO_FLAG_DOWNSTREAM 8u   /* after an event in the same pixel */

typedef struct {
  double R[9]; /* world -> camera rotation, row-major */
  double t[3]; /* world -> camera translation */
  double fx, fy, cx, cy;
  int32_t width, height;
  int32_t pad[2];
} fso_camera;

typedef struct {
  int valid;
  double depth;        /* view-space z of the mean */
  double mx, my;       /* projected mean, pixel units */
  double ca, cb, cc;   /* conic = inverse 2D covariance [[ca cb][cb cc]] */
  double opacity;
  double lno;          /* ln(opacity) */
  int x0, x1, y0, y1;  /* inclusive pixel bounding box of the alpha>=1/255 ellipse */
  /* reduced-precision record (record_f16): alpha = o 2^-|W (p - m)|^2 with
   * the whitening matrix W rounded to FP16 and the mean m rounded to FP32 */
  int f16;
  double w[4];         /* W row-major, each entry an FP16 value */
  double mxr, myr;     /* mean, each an FP32 value */
} fso_proj;

/* ------------------------------------------------------------------------ */
/* Projection (Sec. 3.1: 3D Gaussians are projected to 2D Gaussians          */
/* (m^2D, Sigma^2D) and rendered with the tile rasteriser)                   */
/* ------------------------------------------------------------------------ */

static int project_one(const fso_camera* cam, const float* m, const float* q4,
                       const float* s3, float opac, int record_f16, int coverage, fso_proj* p) {
  p->valid = 0;
  p->f16 = 0;
  const double mx = m[0], my = m[1], mz = m[2];
  const double* R = cam->R;
  const double tx = R[0] * mx + R[1] * my + R[2] * mz + cam->t[0];
  const double ty = R[3] * mx + R[4] * my + R[5] * mz + cam->t[1];
  const double tz = R[6] * mx + R[7] * my + R[8] * mz + cam->t[2];
  if (!(tz > FSO_NEAR_PLANE)) return 0;
  const double o = opac;
  if (!(o >= FSO_ALPHA_MIN)) return 0; /* alpha <= o can never reach 1/255 */

  /* rotation matrix of the unit quaternion (w, x, y, z) */
  double qw = q4[0], qx = q4[1], qy = q4[2], qz = q4[3];
  const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
  if (!(qn > 0.0)) return -1;
  qw /= qn; qx /= qn; qy /= qn; qz /= qn;
  double Rq[3][3];
  Rq[0][0] = 1.0 - 2.0 * (qy * qy + qz * qz);
  Rq[0][1] = 2.0 * (qx * qy - qw * qz);
  Rq[0][2] = 2.0 * (qx * qz + qw * qy);
  Rq[1][0] = 2.0 * (qx * qy + qw * qz);
  Rq[1][1] = 1.0 - 2.0 * (qx * qx + qz * qz);
  Rq[1][2] = 2.0 * (qy * qz - qw * qx);
  Rq[2][0] = 2.0 * (qx * qz - qw * qy);
  Rq[2][1] = 2.0 * (qy * qz + qw * qx);
  Rq[2][2] = 1.0 - 2.0 * (qx * qx + qy * qy);

  /* Sigma3D = Rq diag(s^2) Rq^T */
  const double s2[3] = {(double)s3[0] * s3[0], (double)s3[1] * s3[1], (double)s3[2] * s3[2]};
  double S3[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += Rq[a][k] * s2[k] * Rq[b][k];
      S3[a][b] = acc;
    }

  /* EWA: Sigma2D = J W Sigma3D W^T J^T, W = camera rotation */
  const double limx = 1.3 * (0.5 * cam->width / cam->fx);
  const double limy = 1.3 * (0.5 * cam->height / cam->fy);
  double ux = tx / tz, uy = ty / tz;
  if (ux < -limx) ux = -limx;
  if (ux > limx) ux = limx;
  if (uy < -limy) uy = -limy;
  if (uy > limy) uy = limy;
  const double J[2][3] = {{cam->fx / tz, 0.0, -cam->fx * ux / tz},
                          {0.0, cam->fy / tz, -cam->fy * uy / tz}};
  double T[2][3]; /* T = J W */
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += J[a][k] * R[3 * k + b];
      T[a][b] = acc;
    }
  double S2[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc += T[a][k] * S3[k][l] * T[b][l];
      S2[a][b] = acc;
    }
  const double sa = S2[0][0] + FSO_LOWPASS;
  const double sb = 0.5 * (S2[0][1] + S2[1][0]);
  const double sc = S2[1][1] + FSO_LOWPASS;
  const double det = sa * sc - sb * sb;
  if (!(det > 0.0)) return 0;

  p->depth = tz;
  p->mx = cam->fx * tx / tz + cam->cx;
  p->my = cam->fy * ty / tz + cam->cy;
  p->ca = sc / det;
  p->cb = -sb / det;
  p->cc = sa / det;
  p->opacity = o;
  p->lno = log(o);
  if (record_f16) {
    /* Whitening matrix W with |W d|^2 = 0.5 log2(e) d^T Sigma^-1 d:
     * W = sqrt(0.5 log2 e) diag(lambda1, lambda2)^-1/2 [e1 e2]^T, e1 the unit
     * eigenvector of the larger eigenvalue taken as (h + r, b) for h >= 0 and
     * (b, r - h) otherwise (h = (a - c)/2, r = sqrt(h^2 + b^2)), e2 = e1
     * turned by +90 degrees; then each entry rounded to FP16 and the mean to
     * FP32 (the reduced-precision record). */
    const double h = 0.5 * (sa - sc), rr = sqrt(h * h + sb * sb);
    const double l1 = 0.5 * (sa + sc) + rr, l2 = det / l1;
    double ex, ey;
    if (h >= 0.0) { ex = h + rr; ey = sb; } else { ex = sb; ey = rr - h; }
    const double en = sqrt(ex * ex + ey * ey);
    if (en > 0.0) { ex /= en; ey /= en; } else { ex = 1.0; ey = 0.0; }
    const double k1 = sqrt(FSO_HALF_LOG2E / l1), k2 = sqrt(FSO_HALF_LOG2E / l2);
    p->w[0] = (double)(_Float16)(ex * k1);
    p->w[1] = (double)(_Float16)(ey * k1);
    p->w[2] = (double)(_Float16)(-ey * k2);
    p->w[3] = (double)(_Float16)(ex * k2);
    p->mxr = (double)(float)p->mx;
    p->myr = (double)(float)p->my;
    p->f16 = 1;
  }

  /* alpha >= 1/255 requires d^T C d <= 2 ln(255 o); the ellipse
   * {d : d^T Sigma^-1 d <= r2} has half extents sqrt(Sigma_xx r2),
   * sqrt(Sigma_yy r2).  One pixel of margin. */
  const double r2 = 2.0 * log(255.0 * o);
  const double hx = sqrt(sa * (r2 > 0 ? r2 : 0.0));
  const double hy = sqrt(sc * (r2 > 0 ? r2 : 0.0));
  /* pixel u is sampled at u + 0.5 */
  double fx0 = ceil(p->mx - hx - 0.5 - 1.0), fx1 = floor(p->mx + hx - 0.5 + 1.0);
  double fy0 = ceil(p->my - hy - 0.5 - 1.0), fy1 = floor(p->my + hy - 0.5 + 1.0);
  if (fx0 < 0) fx0 = 0;
  if (fy0 < 0) fy0 = 0;
  if (fx1 > cam->width - 1) fx1 = cam->width - 1;
  if (fy1 > cam->height - 1) fy1 = cam->height - 1;
  if (coverage == FSO_COVERAGE_3SIGMA) {
    /* the standard 3D-GS rasteriser's coverage: the 16x16 tiles that the
     * square of half side r = ceil(3 sqrt(lambda_max(Sigma2D))) around the
     * projected mean overlaps (continuous x in [mx - r, mx + r] against tile
     * t's [16 t, 16 t + 16)); no pixel outside those tiles sees the Gaussian.
     * r and the tiles are integers decided by floating point, so they are
     * decided in the kernel's precision: FP32 from the FP32-rounded 2D
     * covariance and mean, each step rounded to nearest (the library is built
     * without contraction) */
    const float fa = (float)sa, fb = (float)sb, fc = (float)sc;
    const float fmx = (float)p->mx, fmy = (float)p->my;
    const float mid = 0.5f * (fa + fc);
    const float hd = 0.5f * (fa - fc);
    const float lmax = mid + sqrtf(hd * hd + fb * fb);
    const float r = ceilf(3.0f * sqrtf(lmax));
    const float inv = 1.0f / FSO_TILE;
    const double tx0 = floorf((fmx - r) * inv), tx1 = ceilf((fmx + r) * inv) - 1.0f;
    const double ty0 = floorf((fmy - r) * inv), ty1 = ceilf((fmy + r) * inv) - 1.0f;
    if (fx0 < tx0 * FSO_TILE) fx0 = tx0 * FSO_TILE;
    if (fx1 > tx1 * FSO_TILE + (FSO_TILE - 1)) fx1 = tx1 * FSO_TILE + (FSO_TILE - 1);
    if (fy0 < ty0 * FSO_TILE) fy0 = ty0 * FSO_TILE;
    if (fy1 > ty1 * FSO_TILE + (FSO_TILE - 1)) fy1 = ty1 * FSO_TILE + (FSO_TILE - 1);
  }
  if (fx0 > fx1 || fy0 > fy1) return 0;
  p->x0 = (int)fx0; p->x1 = (int)fx1; p->y0 = (int)fy0; p->y1 = (int)fy1;
  p->valid = 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One pixel: front-to-back compositing (Eq. 1)                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t g;       /* Gaussian index */
  double c;        /* alpha * T added by the oracle (0 if not added) */
  double risk;     /* bound on |change of c| if a marginal decision flips */
  uint8_t flag;    /* event flags raised at this pixel for g */
} fso_hit;

/* Walk the candidate list `cand` (length n, already in (depth, index) order)
 * for the pixel centred at (px, py), Eq. 1 term by term.  Writes every
 * contribution into `hits` (capacity >= n) and returns how many; *t_final
 * receives the transmittance left when the walk ends.
 *
 * Discrete decisions that sit within a small relative window of their
 * threshold (alpha vs 1/255, T(1-alpha) vs 1e-4, equal depths) are ones an
 * implementation with other rounding may take the other way.  For them the
 * walk records, per Gaussian, `risk`: an upper bound on how much that
 * Gaussian's alpha*T at this pixel changes if the decision flips.  Gaussians
 * the oracle does not add but another walk could are listed with c = 0.
 * `use_bbox` skips candidates whose pixel bounding box excludes the pixel. */
static int walk_pixel(const fso_proj* P, const int32_t* cand, int64_t n, int use_bbox,
                      int px_i, int py_i, const fso_rule* rule, double depth_limit, fso_hit* hits,
                      double* t_final, int64_t* n_eval, int64_t* n_part) {
  const double px = px_i + 0.5, py = py_i + 0.5;
  const double ev_rel = rule->ev_rel, a_min = rule->alpha_min, t_min = rule->t_min;
  /* ln of the smallest alpha any branch below looks at: a candidate under it
   * is skipped before its exponential is taken (the same decision) */
  const double ln_floor = log(a_min * (1.0 - ev_rel)) - 1e-9;
  double T = 1.0;
  double sa = 0.0;        /* sum of alpha/(1 - alpha) over the factors of T so far */
  int64_t n_fac = 0;      /* factors of T so far */
  int nh = 0;
  double down = 0.0;      /* relative uncertainty of T from earlier marginal events */
  int all_risky = 0;      /* a marginal stop was passed: every later term may change */
  int stopped = 0;        /* the oracle stopped on a marginal test; T_shadow continues */
  double T_shadow = 0.0;
  int last_hit = -1;
  for (int64_t k = 0; k < n; ++k) {
    const int32_t g = cand[k];
    const fso_proj* p = &P[g];
    if (p->depth > depth_limit) break; /* nothing tracked lies further back */
    if (use_bbox && (px_i < p->x0 || px_i > p->x1 || py_i < p->y0 || py_i > p->y1)) continue;
    ++*n_eval;
    double alpha;
    if (p->f16) {
      const double dx = px - p->mxr, dy = py - p->myr;
      const double w0 = p->w[0] * dx + p->w[1] * dy, w1 = p->w[2] * dx + p->w[3] * dy;
      const double q = w0 * w0 + w1 * w1;
      if (p->lno - q * 0.69314718055994530942 < ln_floor) continue;
      alpha = p->opacity * exp2(-q);
    } else {
      const double dx = px - p->mx, dy = py - p->my;
      const double power = -0.5 * (p->ca * dx * dx + p->cc * dy * dy) - p->cb * dx * dy;
      if (p->lno + power < ln_floor) continue;
      alpha = p->opacity * exp(power);
    }
    if (alpha > FSO_ALPHA_MAX) alpha = FSO_ALPHA_MAX;
    const int a_edge = fabs(alpha - a_min) <= ev_rel * a_min;
    if (stopped) {
      /* Beyond a marginal stop: another walk may keep adding terms. */
      if (alpha >= a_min * (1.0 - ev_rel)) {
        hits[nh].g = g; hits[nh].c = 0.0;
        hits[nh].risk = alpha * T_shadow * (1.0 + down) + 1e-300;
        hits[nh].flag = FSO_FLAG_DOWNSTREAM | (a_edge ? FSO_FLAG_ALPHA_EDGE : 0);
        ++nh;
        T_shadow *= 1.0 - alpha;
      }
      continue;
    }
    if (alpha < a_min) {
      if (a_edge) { /* skipped here, but on the threshold: another walk may add it */
        hits[nh].g = g; hits[nh].c = 0.0;
        hits[nh].risk = alpha * T * (1.0 + down);
        hits[nh].flag = FSO_FLAG_ALPHA_EDGE;
        ++nh;
        down += alpha / (1.0 - alpha);
      }
      continue;
    }
    ++*n_part; /* alpha >= 1/255 before the stop: this pair takes part (the stop included) */
    const double test_T = T * (1.0 - alpha);
    /* the relative error another implementation's test_T may carry: alpha's
     * relative error carried through every factor, each factor's rounding,
     * and the uncertainty `down` of T after marginal alpha decisions earlier
     * in this pixel */
    const double t_win = ev_rel * (1.0 + sa + alpha / (1.0 - alpha)) +
                         (double)(n_fac + 1) * 0x1p-23 + 1.01 * down;
    const int t_edge = fabs(test_T - t_min) <= t_win * t_min;
    if (test_T < t_min) {
      if (t_edge || all_risky) {
        /* the stop may not happen in another walk: this term and all
         * later ones are at risk */
        hits[nh].g = g; hits[nh].c = 0.0;
        hits[nh].risk = alpha * T * (1.0 + down);
        hits[nh].flag = FSO_FLAG_T_EDGE;
        ++nh;
        stopped = 1;
        T_shadow = test_T;
        continue;
      }
      break;
    }
    const double c = alpha * T;
    double risk = c * down;
    uint8_t fl = down > 0.0 ? FSO_FLAG_DOWNSTREAM : 0;
    if (a_edge) { risk = c * (1.0 + down); fl |= FSO_FLAG_ALPHA_EDGE; }
    if (t_edge || all_risky) { risk = c * (1.0 + down); fl |= FSO_FLAG_T_EDGE; all_risky = 1; }
    if (last_hit >= 0 &&
        fabs(p->depth - P[hits[last_hit].g].depth) <= FSO_DEPTH_TIE_REL * p->depth) {
      /* swapping two neighbours changes each term by alpha_a*alpha_b*T */
      const double swap = hits[last_hit].c * alpha; /* alpha_a alpha_b T_before */
      risk += swap;
      hits[last_hit].risk += swap;
      fl |= FSO_FLAG_DEPTH_TIE;
      hits[last_hit].flag |= FSO_FLAG_DEPTH_TIE;
    }
    hits[nh].g = g; hits[nh].c = c; hits[nh].risk = risk; hits[nh].flag = fl;
    last_hit = nh;
    ++nh;
    if (a_edge) down += alpha / (1.0 - alpha);
    sa += alpha / (1.0 - alpha);
    ++n_fac;
    T = test_T;
  }
  *t_final = T;
  return nh;
}

/* ------------------------------------------------------------------------ */
/* Per-view setup: projection, depth order, spatial bins                     */
/* ------------------------------------------------------------------------ */

static const fso_proj* g_sort_P; /* qsort has no context argument in C99 */
static int g_tie_reverse;        /* equal depths by higher index first (tests only) */

static int cmp_depth(const void* a, const void* b) {
  const int32_t ia = *(const int32_t*)a, ib = *(const int32_t*)b;
  const double da = g_sort_P[ia].depth, db = g_sort_P[ib].depth;
  if (da < db) return -1;
  if (da > db) return 1;
  return g_tie_reverse ? (ia < ib) - (ia > ib) : (ia > ib) - (ia < ib);
}

typedef struct {
  int64_t N;
  const float *mean, *quat, *scale, *opacity;
  const fso_camera* cam;
  fso_proj* P;
  int64_t begin, end;
  int record_f16;
  int coverage;
  int status;
} proj_job;

static void* proj_worker(void* arg) {
  proj_job* j = (proj_job*)arg;
  for (int64_t i = j->begin; i < j->end; ++i) {
    if (project_one(j->cam, j->mean + 3 * i, j->quat + 4 * i, j->scale + 3 * i, j->opacity[i],
                    j->record_f16, j->coverage, &j->P[i]) < 0)
      j->status = -1;
  }
  return NULL;
}

typedef struct {
  int32_t* order;  /* valid Gaussians in (depth, index) order */
  int64_t n_valid;
  int bins_x, bins_y;
  int64_t* bin_start; /* [bins+1] */
  int32_t* bin_list;  /* Gaussians per bin, each bin in depth order */
} view_index;

/* Projects all N Gaussians into the view (threads over index ranges). */
static int project_all(int64_t N, const float* mean, const float* quat, const float* scale,
                       const float* opacity, const fso_camera* cam, int nthreads, int record_f16,
                       int coverage, fso_proj* P) {
  if (nthreads < 1) nthreads = 1;
  proj_job* jobs = (proj_job*)calloc((size_t)nthreads, sizeof(proj_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (proj_job){N, mean, quat, scale, opacity, cam, P, N * t / nthreads,
                         N * (t + 1) / nthreads, record_f16, coverage, 0};
    pthread_create(&th[t], NULL, proj_worker, &jobs[t]);
  }
  int status = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].status) status = jobs[t].status;
  }
  free(jobs);
  free(th);
  return status;
}

/* Depth order and spatial bins of the projected Gaussians P.  rect
 * (x0, x1, y0, y1) or NULL: only Gaussians whose pixel bounding box meets the
 * rect are indexed (the others cannot reach a pixel inside it).  member or
 * NULL: only Gaussians i with member[i] & member_bit are indexed. */
static int index_view(int64_t N, const fso_camera* cam, const fso_proj* P, int build_bins,
                      const int* rect, const uint64_t* member, uint64_t member_bit,
                      view_index* vi) {
  memset(vi, 0, sizeof(*vi));
  int64_t nv = 0;
  for (int64_t i = 0; i < N; ++i) nv += P[i].valid;
  vi->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
  nv = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (!P[i].valid) continue;
    if (member && !(member[i] & member_bit)) continue;
    if (rect && (P[i].x1 < rect[0] || P[i].x0 > rect[1] || P[i].y1 < rect[2] || P[i].y0 > rect[3]))
      continue;
    vi->order[nv++] = (int32_t)i;
  }
  vi->n_valid = nv;
  g_sort_P = P;
  qsort(vi->order, (size_t)nv, sizeof(int32_t), cmp_depth);

  if (!build_bins) return 0;
  const int bx = (cam->width + FSO_BIN - 1) / FSO_BIN, by = (cam->height + FSO_BIN - 1) / FSO_BIN;
  vi->bins_x = bx;
  vi->bins_y = by;
  int64_t nb = (int64_t)bx * by;
  vi->bin_start = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
  for (int64_t k = 0; k < nv; ++k) {
    const fso_proj* p = &P[vi->order[k]];
    for (int y = p->y0 / FSO_BIN; y <= p->y1 / FSO_BIN; ++y)
      for (int x = p->x0 / FSO_BIN; x <= p->x1 / FSO_BIN; ++x) vi->bin_start[(int64_t)y * bx + x + 1]++;
  }
  for (int64_t b = 0; b < nb; ++b) vi->bin_start[b + 1] += vi->bin_start[b];
  vi->bin_list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(vi->bin_start[nb] > 0 ? vi->bin_start[nb] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
  memcpy(fill, vi->bin_start, sizeof(int64_t) * (size_t)nb);
  for (int64_t k = 0; k < nv; ++k) { /* depth order is kept inside each bin */
    const int32_t g = vi->order[k];
    const fso_proj* p = &P[g];
    for (int y = p->y0 / FSO_BIN; y <= p->y1 / FSO_BIN; ++y)
      for (int x = p->x0 / FSO_BIN; x <= p->x1 / FSO_BIN; ++x) vi->bin_list[fill[(int64_t)y * bx + x]++] = g;
  }
  free(fill);
  return 0;
}

static void free_view(view_index* vi) {
  free(vi->order);
  free(vi->bin_start);
  free(vi->bin_list);
  memset(vi, 0, sizeof(*vi));
}

/* ------------------------------------------------------------------------ */
/* Accumulation of the contribution table (Eq. 6 / Eq. 7)                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  /* shared, read-only */
  const fso_proj* P;
  const view_index* vi;
  const fso_camera* cam;
  const int32_t* mask;      /* this view's labels, row-major H x W */
  const int64_t* slot;      /* Gaussian -> table row, -1 = not tracked */
  const uint8_t* pix_sel;   /* NULL or per-pixel "walk this pixel" */
  int32_t E;
  int cull_mode;
  int coverage;
  const fso_rule* rule;     /* thresholds and near-threshold window */
  double depth_limit;       /* walks end beyond this depth (tracked rows only) */
  int nthreads, tid;
  double* t_final;          /* this view's slice or NULL */
  /* per thread */
  double* table;            /* [rows][E] */
  double* risk;             /* [rows][E] */
  uint8_t* flags;           /* [rows] */
  fso_hit* hits;            /* scratch, capacity max candidates */
  int64_t n_eval, n_hit, n_bad, n_part;
} acc_job;

static void* acc_worker(void* arg) {
  acc_job* j = (acc_job*)arg;
  const int W = j->cam->width, H = j->cam->height;
  for (int y = j->tid; y < H; y += j->nthreads) {
    for (int x = 0; x < W; ++x) {
      const int64_t pix = (int64_t)y * W + x;
      if (j->pix_sel && !j->pix_sel[pix]) continue;
      const int32_t* cand;
      int64_t n;
      if (j->cull_mode == 1) {
        cand = j->vi->order;
        n = j->vi->n_valid;
      } else {
        const int64_t b = (int64_t)(y / FSO_BIN) * j->vi->bins_x + x / FSO_BIN;
        cand = j->vi->bin_list + j->vi->bin_start[b];
        n = j->vi->bin_start[b + 1] - j->vi->bin_start[b];
      }
      double tf;
      const int nh = walk_pixel(j->P, cand, n, j->cull_mode != 1 || j->coverage != 0, x, y, j->rule,
                                j->depth_limit, j->hits, &tf, &j->n_eval, &j->n_part);
      if (j->t_final) j->t_final[pix] = tf;
      const int32_t lab = j->mask[pix];
      const int lab_ok = (lab >= 0 && lab < j->E);
      if (!lab_ok) j->n_bad++;
      for (int h = 0; h < nh; ++h) {
        const int64_t r = j->slot ? j->slot[j->hits[h].g] : j->hits[h].g;
        if (r < 0) continue;
        if (j->hits[h].c > 0.0) j->n_hit++;
        j->flags[r] |= j->hits[h].flag;
        if (lab_ok) {
          j->table[r * j->E + lab] += j->hits[h].c;
          j->risk[r * j->E + lab] += j->hits[h].risk;
        }
      }
    }
  }
  return NULL;
}

/* Tracked rows (sel): each tracked Gaussian g is handled on its own, per
 * view.  Its candidates are the Gaussians whose bounding box meets g's (found
 * through a coarse grid of the view), in (depth, index) order -- every
 * Gaussian that covers a pixel of g's box is among them -- and only the
 * pixels of g's box are walked, adding only g's terms.  Row r belongs to thread r % nthreads, so each row's sum has a fixed
 * order. */
typedef struct {
  const fso_proj* P;
  int64_t N;
  const fso_camera* cam;
  const int32_t* mask;
  const int64_t* sel;
  int64_t n_sel;
  int32_t E;
  const fso_rule* rule;
  const int64_t* cell_start; /* coarse grid of the view: Gaussians per cell */
  const int32_t* cell_list;
  int cells_x, cells_y;
  uint32_t* stamp;           /* per Gaussian: last tracked row that listed it */
  int nthreads, tid;
  double* table;            /* [rows][E], this thread's rows only */
  double* risk;
  uint8_t* flags;
  int32_t* cand;            /* capacity N */
  fso_hit* hits;            /* capacity N */
  fso_proj* local;          /* the candidates' records, in depth order (grown as needed) */
  int64_t local_cap;
  int64_t n_eval, n_hit, n_bad, n_part;
} sel_job;

static void* sel_worker(void* arg) {
  sel_job* j = (sel_job*)arg;
  const fso_proj* P = j->P;
  const int W = j->cam->width;
  for (int64_t r = j->tid; r < j->n_sel; r += j->nthreads) {
    const int32_t g = (int32_t)j->sel[r];
    const fso_proj* pg = &P[g];
    if (!pg->valid) continue;
    /* candidates: the Gaussians listed in the grid cells g's box meets
     * whose own box meets g's (each taken once) */
    int64_t nc = 0;
    const uint32_t tag = (uint32_t)r + 1u;
    const int cx0 = pg->x0 / FSO_CELL, cx1 = pg->x1 / FSO_CELL;
    const int cy0 = pg->y0 / FSO_CELL, cy1 = pg->y1 / FSO_CELL;
    for (int cy = cy0; cy <= cy1; ++cy)
      for (int cx = cx0; cx <= cx1; ++cx) {
        const int64_t c = (int64_t)cy * j->cells_x + cx;
        for (int64_t k = j->cell_start[c]; k < j->cell_start[c + 1]; ++k) {
          const int32_t i = j->cell_list[k];
          if (j->stamp[i] == tag) continue;
          j->stamp[i] = tag;
          const fso_proj* q = &P[i];
          if (!(q->x1 < pg->x0 || q->x0 > pg->x1 || q->y1 < pg->y0 || q->y0 > pg->y1))
            j->cand[nc++] = i;
        }
      }
    qsort(j->cand, (size_t)nc, sizeof(int32_t), cmp_depth);
    /* the candidates' records side by side in depth order: the walks below
     * read them from this local copy (local index k is candidate k) */
    if (nc > j->local_cap) {
      free(j->local);
      j->local_cap = nc + nc / 2 + 1024;
      j->local = (fso_proj*)malloc(sizeof(fso_proj) * (size_t)j->local_cap);
    }
    for (int64_t k = 0; k < nc; ++k) j->local[k] = P[j->cand[k]];
    int64_t g_local = -1;
    for (int64_t k = 0; k < nc; ++k)
      if (j->cand[k] == g) g_local = k;
    /* 8x8-pixel bins over g's box, each holding its candidates in order */
    const int nbx = (pg->x1 - pg->x0) / FSO_BIN + 1, nby = (pg->y1 - pg->y0) / FSO_BIN + 1;
    const int64_t nb = (int64_t)nbx * nby;
    int64_t* start = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
    for (int64_t k = 0; k < nc; ++k) {
      const fso_proj* q = &j->local[k];
      const int bx0 = ((q->x0 > pg->x0 ? q->x0 : pg->x0) - pg->x0) / FSO_BIN;
      const int bx1 = ((q->x1 < pg->x1 ? q->x1 : pg->x1) - pg->x0) / FSO_BIN;
      const int by0 = ((q->y0 > pg->y0 ? q->y0 : pg->y0) - pg->y0) / FSO_BIN;
      const int by1 = ((q->y1 < pg->y1 ? q->y1 : pg->y1) - pg->y0) / FSO_BIN;
      for (int by = by0; by <= by1; ++by)
        for (int bx = bx0; bx <= bx1; ++bx) start[(int64_t)by * nbx + bx + 1]++;
    }
    for (int64_t b = 0; b < nb; ++b) start[b + 1] += start[b];
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(start[nb] > 0 ? start[nb] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    memcpy(fill, start, sizeof(int64_t) * (size_t)nb);
    for (int64_t k = 0; k < nc; ++k) {
      const fso_proj* q = &j->local[k];
      const int bx0 = ((q->x0 > pg->x0 ? q->x0 : pg->x0) - pg->x0) / FSO_BIN;
      const int bx1 = ((q->x1 < pg->x1 ? q->x1 : pg->x1) - pg->x0) / FSO_BIN;
      const int by0 = ((q->y0 > pg->y0 ? q->y0 : pg->y0) - pg->y0) / FSO_BIN;
      const int by1 = ((q->y1 < pg->y1 ? q->y1 : pg->y1) - pg->y0) / FSO_BIN;
      for (int by = by0; by <= by1; ++by)
        for (int bx = bx0; bx <= bx1; ++bx) list[fill[(int64_t)by * nbx + bx]++] = (int32_t)k;
    }
    free(fill);
    /* a walk can end past g: later Gaussians do not change earlier terms
     * (the margin keeps exact depth ties with g inside the walk) */
    const double depth_limit = pg->depth * (1.0 + 1e-9);
    for (int y = pg->y0; y <= pg->y1; ++y) {
      for (int x = pg->x0; x <= pg->x1; ++x) {
        double tf;
        const int64_t b = (int64_t)((y - pg->y0) / FSO_BIN) * nbx + (x - pg->x0) / FSO_BIN;
        const int nh = walk_pixel(j->local, list + start[b], start[b + 1] - start[b], 1, x, y,
                                  j->rule, depth_limit, j->hits, &tf, &j->n_eval, &j->n_part);
        const int32_t lab = j->mask[(int64_t)y * W + x];
        const int lab_ok = (lab >= 0 && lab < j->E);
        if (!lab_ok) j->n_bad++;
        for (int h = 0; h < nh; ++h) {
          if (j->hits[h].g != g_local) continue;
          if (j->hits[h].c > 0.0) j->n_hit++;
          j->flags[r] |= j->hits[h].flag;
          if (lab_ok) {
            j->table[r * j->E + lab] += j->hits[h].c;
            j->risk[r * j->E + lab] += j->hits[h].risk;
          }
        }
      }
    }
    free(start);
    free(list);
  }
  return NULL;
}

/*
 * fso_accumulate: fill table[rows][E] (FP64) with the per-label contribution
 * sums of Eq. 6/7 over all V views, and risk[rows][E] with the summed bounds
 * on how much each entry moves if marginal decisions flip (see walk_pixel).
 *
 *   mean[N*3], quat[N*4] (w,x,y,z), scale[N*3] (linear), opacity[N] (activated)
 *   cams[V]; masks: view v's int32 labels at masks + mask_offsets[v] (H*W)
 *   sel: NULL -> rows = N, row i = Gaussian i; otherwise n_sel sorted Gaussian
 *        indices and only those rows are tracked (each is walked on its own
 *        over its bounding box; see sel_worker -- the rows do not change)
 *   cull_mode: 0 = spatial bins, 1 = every pixel walks every Gaussian
 *   t_final: NULL or [sum_v H*W] transmittance left at each pixel (-1 where
 *        the pixel was not walked); only without sel
 *   stats[5]: evaluated pairs (candidates in the pixel's walk up to its stop),
 *        contributing pairs (alpha*T added), pixels with bad labels, tracked
 *        Gaussians that were never valid in any view, and the pairs that take
 *        part in the compositing (alpha >= 1/255, up to and including the
 *        stop; without sel only)
 *   event_rel: the relative precision assumed for alpha, which sets the
 *        windows of the near-threshold model above (<= 0: FSO_EVENT_REL)
 *   record_f16: non-zero -> alpha from the reduced-precision record (FP16
 *        whitening matrix, FP32 mean; see fso_proj), all else unchanged
 *   alpha_min, t_min: the rule's thresholds (<= 0: 1/255 and 1e-4); tests
 *        move them inside their windows
 *   tie_reverse: non-zero -> equal depths are walked by higher index first
 *   coverage: 0 = every pixel the alpha >= 1/255 ellipse reaches (exact);
 *        FSO_COVERAGE_3SIGMA = only pixels in the 16x16 tiles of the 3-sigma
 *        square (the standard rasteriser's tile coverage)
 * Returns 0, or -1 on a zero quaternion, -2 on bad arguments.
 */
int fso_accumulate(int64_t N, const float* mean, const float* quat, const float* scale,
                   const float* opacity, int32_t V, const fso_camera* cams,
                   const int32_t* masks, const int64_t* mask_offsets, int32_t E,
                   const int64_t* sel, int64_t n_sel, int32_t cull_mode, int32_t nthreads,
                   double* table, double* risk, uint8_t* flags, double* t_final,
                   int64_t* stats, double event_rel, int32_t record_f16, double alpha_min,
                   double t_min, int32_t tie_reverse, int32_t coverage) {
  if (N < 0 || V < 0 || E < 1 || (sel && n_sel < 0)) return -2;
  if (sel && t_final) return -2;
  fso_rule rule;
  rule.ev_rel = event_rel > 0.0 ? event_rel : FSO_EVENT_REL;
  rule.alpha_min = alpha_min > 0.0 ? alpha_min : FSO_ALPHA_MIN;
  rule.t_min = t_min > 0.0 ? t_min : FSO_T_MIN;
  g_tie_reverse = tie_reverse != 0;
  if (nthreads < 1) nthreads = 1;
  const int64_t rows = sel ? n_sel : N;
  int64_t* slot = NULL;
  if (sel) {
    slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) slot[i] = -1;
    for (int64_t r = 0; r < n_sel; ++r) {
      if (sel[r] < 0 || sel[r] >= N) { free(slot); return -2; }
      slot[sel[r]] = r;
    }
  }
  memset(table, 0, sizeof(double) * (size_t)(rows * E));
  memset(risk, 0, sizeof(double) * (size_t)(rows * E));
  memset(flags, 0, (size_t)rows);
  int64_t st[5] = {0, 0, 0, 0, 0};

  fso_proj* P = (fso_proj*)malloc(sizeof(fso_proj) * (size_t)(N > 0 ? N : 1));
  acc_job* jobs = (acc_job*)calloc((size_t)nthreads, sizeof(acc_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].table = (double*)calloc((size_t)(rows * E > 0 ? rows * E : 1), sizeof(double));
    jobs[t].risk = (double*)calloc((size_t)(rows * E > 0 ? rows * E : 1), sizeof(double));
    jobs[t].flags = (uint8_t*)calloc((size_t)(rows > 0 ? rows : 1), 1);
  }
  uint8_t* seen = (uint8_t*)calloc((size_t)(rows > 0 ? rows : 1), 1);
  int status = 0;
  int64_t pix_base = 0;
  for (int32_t v = 0; v < V && !status; ++v) {
    const fso_camera* cam = &cams[v];
    const int64_t npix = (int64_t)cam->width * cam->height;
    view_index vi;
    status = project_all(N, mean, quat, scale, opacity, cam, nthreads, record_f16, coverage, P);
    if (status) break;
    if (sel) {
      int any = 0;
      for (int64_t r = 0; r < n_sel; ++r)
        if (P[sel[r]].valid) seen[r] = any = 1;
      if (any) {
        g_sort_P = P;
        /* coarse grid of the view: every valid Gaussian listed in the
         * 32x32-pixel cells its box meets */
        const int gcx = (cam->width + FSO_CELL - 1) / FSO_CELL;
        const int gcy = (cam->height + FSO_CELL - 1) / FSO_CELL;
        const int64_t ncell = (int64_t)gcx * gcy;
        int64_t* cstart = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
        for (int64_t i = 0; i < N; ++i) {
          if (!P[i].valid) continue;
          for (int cy = P[i].y0 / FSO_CELL; cy <= P[i].y1 / FSO_CELL; ++cy)
            for (int cx = P[i].x0 / FSO_CELL; cx <= P[i].x1 / FSO_CELL; ++cx)
              cstart[(int64_t)cy * gcx + cx + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
        int32_t* clist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cstart[ncell] > 0 ? cstart[ncell] : 1));
        int64_t* cfill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell > 0 ? ncell : 1));
        memcpy(cfill, cstart, sizeof(int64_t) * (size_t)ncell);
        for (int64_t i = 0; i < N; ++i) {
          if (!P[i].valid) continue;
          for (int cy = P[i].y0 / FSO_CELL; cy <= P[i].y1 / FSO_CELL; ++cy)
            for (int cx = P[i].x0 / FSO_CELL; cx <= P[i].x1 / FSO_CELL; ++cx)
              clist[cfill[(int64_t)cy * gcx + cx]++] = (int32_t)i;
        }
        free(cfill);
        sel_job* sj = (sel_job*)calloc((size_t)nthreads, sizeof(sel_job));
        for (int t = 0; t < nthreads; ++t) {
          sj[t] = (sel_job){P, N, cam, masks + mask_offsets[v], sel, n_sel, E, &rule,
                            cstart, clist, gcx, gcy,
                            (uint32_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(uint32_t)),
                            nthreads, t, jobs[t].table, jobs[t].risk, jobs[t].flags,
                            (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1)),
                            (fso_hit*)malloc(sizeof(fso_hit) * (size_t)(N > 0 ? N : 1)), NULL,
                            0, 0, 0, 0, 0};
          pthread_create(&th[t], NULL, sel_worker, &sj[t]);
        }
        for (int t = 0; t < nthreads; ++t) {
          pthread_join(th[t], NULL);
          jobs[t].n_eval += sj[t].n_eval;
          jobs[t].n_hit += sj[t].n_hit;
          jobs[t].n_bad += sj[t].n_bad;
          free(sj[t].cand);
          free(sj[t].hits);
          free(sj[t].local);
          free(sj[t].stamp);
        }
        free(sj);
        free(cstart);
        free(clist);
      }
      pix_base += npix;
      continue;
    }
    status = index_view(N, cam, P, cull_mode != 1, NULL, NULL, 0, &vi);
    if (status) { free_view(&vi); break; }
    for (int64_t i = 0; i < N; ++i)
      if (P[i].valid) seen[i] = 1;
    uint8_t* pix_sel = NULL;
    if (t_final) {
      for (int64_t k = 0; k < npix; ++k) t_final[pix_base + k] = -1.0;
    }
    /* the longest candidate list bounds the hits of one pixel */
    int64_t max_cand = vi.n_valid;
    if (cull_mode != 1) {
      max_cand = 0;
      const int64_t nb = (int64_t)vi.bins_x * vi.bins_y;
      for (int64_t b = 0; b < nb; ++b) {
        const int64_t c = vi.bin_start[b + 1] - vi.bin_start[b];
        if (c > max_cand) max_cand = c;
      }
    }
    for (int t = 0; t < nthreads; ++t) {
      acc_job* j = &jobs[t];
      j->P = P; j->vi = &vi; j->cam = cam; j->mask = masks + mask_offsets[v];
      j->slot = slot; j->pix_sel = pix_sel; j->E = E; j->cull_mode = cull_mode;
      j->coverage = coverage;
      j->rule = &rule;
      j->depth_limit = INFINITY;
      j->nthreads = nthreads; j->tid = t;
      j->t_final = t_final ? t_final + pix_base : NULL;
      j->hits = (fso_hit*)malloc(sizeof(fso_hit) * (size_t)(max_cand > 0 ? max_cand : 1));
      pthread_create(&th[t], NULL, acc_worker, j);
    }
    for (int t = 0; t < nthreads; ++t) {
      pthread_join(th[t], NULL);
      free(jobs[t].hits);
      jobs[t].hits = NULL;
    }
    free(pix_sel);
    free_view(&vi);
    pix_base += npix;
  }
  /* fixed-order merge of the per-thread partial tables */
  for (int t = 0; t < nthreads; ++t) {
    for (int64_t k = 0; k < rows * E; ++k) table[k] += jobs[t].table[k];
    for (int64_t k = 0; k < rows * E; ++k) risk[k] += jobs[t].risk[k];
    for (int64_t r = 0; r < rows; ++r) flags[r] |= jobs[t].flags[r];
    st[0] += jobs[t].n_eval;
    st[1] += jobs[t].n_hit;
    st[2] += jobs[t].n_bad;
    st[4] += jobs[t].n_part;
    free(jobs[t].table);
    free(jobs[t].risk);
    free(jobs[t].flags);
  }
  for (int64_t r = 0; r < rows; ++r) st[3] += !seen[r];
  if (stats) memcpy(stats, st, sizeof(st));
  free(seen);
  free(jobs);
  free(th);
  free(P);
  free(slot);
  g_tie_reverse = 0;
  return status;
}

/*
 * fso_pixel_lists: every pixel's ordered list of (Gaussian, alpha*T) -- the
 * terms of Eq. 1 -- for small scenes (brute-force and linearity tests).
 *   pix_offsets[P+1] (CSR over all pixels of all views, views in order,
 *   row-major), gidx/contrib[capacity], t_final[P].
 * Only contributions with alpha*T > 0 are listed.  Returns the number of
 * pairs; when it exceeds `capacity` nothing beyond capacity is written and
 * the caller repeats with a larger buffer.  Negative on error.
 */
int64_t fso_pixel_lists(int64_t N, const float* mean, const float* quat, const float* scale,
                        const float* opacity, int32_t V, const fso_camera* cams,
                        int32_t cull_mode, int64_t capacity, int64_t* pix_offsets,
                        int32_t* gidx, double* contrib, double* t_final) {
  fso_proj* P = (fso_proj*)malloc(sizeof(fso_proj) * (size_t)(N > 0 ? N : 1));
  fso_hit* hits = (fso_hit*)malloc(sizeof(fso_hit) * (size_t)(N > 0 ? N : 1));
  int64_t total = 0, pix = 0, n_eval = 0, n_part = 0;
  const fso_rule rule = {FSO_ALPHA_MIN, FSO_T_MIN, FSO_EVENT_REL};
  for (int32_t v = 0; v < V; ++v) {
    const fso_camera* cam = &cams[v];
    view_index vi;
    int st = project_all(N, mean, quat, scale, opacity, cam, 1, 0, 0, P);
    if (st == 0) st = index_view(N, cam, P, cull_mode != 1, NULL, NULL, 0, &vi);
    if (st) { free_view(&vi); free(P); free(hits); return -1; }
    for (int y = 0; y < cam->height; ++y)
      for (int x = 0; x < cam->width; ++x) {
        const int32_t* cand;
        int64_t n;
        if (cull_mode == 1) {
          cand = vi.order; n = vi.n_valid;
        } else {
          const int64_t b = (int64_t)(y / FSO_BIN) * vi.bins_x + x / FSO_BIN;
          cand = vi.bin_list + vi.bin_start[b];
          n = vi.bin_start[b + 1] - vi.bin_start[b];
        }
        double tf;
        const int nh = walk_pixel(P, cand, n, cull_mode != 1, x, y, &rule, INFINITY,
                                hits, &tf, &n_eval, &n_part);
        pix_offsets[pix] = total;
        if (t_final) t_final[pix] = tf;
        for (int h = 0; h < nh; ++h) {
          if (!(hits[h].c > 0.0)) continue;
          if (total < capacity) {
            gidx[total] = hits[h].g;
            contrib[total] = hits[h].c;
          }
          ++total;
        }
        ++pix;
      }
    free_view(&vi);
  }
  pix_offsets[pix] = total;
  free(P);
  free(hits);
  return total;
}

/*
 * fso_project_view: the projected quantities of one view, for closed-form
 * tests of the projection.  out[N*10] per Gaussian: valid, depth, mx, my,
 * conic a, b, c, opacity, bbox width, bbox height (0 when invalid).
 */
int fso_project_view(int64_t N, const float* mean, const float* quat, const float* scale,
                     const float* opacity, const fso_camera* cam, double* out) {
  for (int64_t i = 0; i < N; ++i) {
    fso_proj p;
    memset(&p, 0, sizeof(p));
    if (project_one(cam, mean + 3 * i, quat + 4 * i, scale + 3 * i, opacity[i], 0, 0, &p) < 0)
      return -1;
    double* o = out + 10 * i;
    o[0] = p.valid;
    o[1] = p.depth; o[2] = p.mx; o[3] = p.my;
    o[4] = p.ca; o[5] = p.cb; o[6] = p.cc; o[7] = p.opacity;
    o[8] = p.valid ? (double)(p.x1 - p.x0 + 1) : 0.0;
    o[9] = p.valid ? (double)(p.y1 - p.y0 + 1) : 0.0;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Novel-view mask rendering (Sec. 3.4; Supp. Sec. 8.2)                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  const fso_proj* P;
  const view_index* vi;     /* the object's Gaussians only */
  const fso_camera* cam;
  int coverage;
  const fso_rule* rule;
  int nthreads, tid;
  double *rho, *z, *rho_risk, *z_risk; /* this object's planes of the view, H*W each */
  fso_hit* hits;
} render_job;

static void* render_worker(void* arg) {
  render_job* j = (render_job*)arg;
  const int W = j->cam->width, H = j->cam->height;
  for (int y = j->tid; y < H; y += j->nthreads) {
    for (int x = 0; x < W; ++x) {
      const int64_t b = (int64_t)(y / FSO_BIN) * j->vi->bins_x + x / FSO_BIN;
      const int32_t* cand = j->vi->bin_list + j->vi->bin_start[b];
      const int64_t n = j->vi->bin_start[b + 1] - j->vi->bin_start[b];
      double tf;
      int64_t n_eval = 0, n_part = 0;
      const int nh = walk_pixel(j->P, cand, n, 1, x, y, j->rule, INFINITY, j->hits, &tf,
                                &n_eval, &n_part);
      double rho = 0.0, z = 0.0, rr = 0.0, zr = 0.0;
      for (int h = 0; h < nh; ++h) {
        const double d = j->P[j->hits[h].g].depth;
        rho += j->hits[h].c;
        z += j->hits[h].c * d;
        rr += j->hits[h].risk;
        zr += j->hits[h].risk * d;
      }
      const int64_t pix = (int64_t)y * W + x;
      j->rho[pix] = rho;
      j->z[pix] = z;
      j->rho_risk[pix] = rr;
      j->z_risk[pix] = zr;
    }
  }
  return NULL;
}

/*
 * fso_render_masks: 2D masks for (novel) views from a segmentation.  Object
 * e = 1 .. E-1 is the subset {G_i}_e = {i : bit e of member[i] set}; each is
 * rendered on its own (Eq. 1 over its Gaussians only, same rules as the
 * accumulation): rho^e = sum alpha T at every pixel, and its depth
 * D^e = sum alpha T z / rho^e, z the view-space depth of the Gaussian's mean
 * (the alpha-weighted depth of Eq. 1 with x_i = z_i, divided by rho^e so it
 * is a depth; 0 where rho^e = 0).  A pixel's mask value is the object with
 * rho^e > tau of smallest D^e (equal depths: the smaller e), else 0 (Sec.
 * 3.4: quantisation at tau, then depth guidance).  With E = 2 this is the
 * binary rule M = [rho^1 > tau].
 *   member[N]: membership bits (bit e: object e); E in [2, 64]
 *   per view v, pixel block at off[v] (sum of earlier views' H*W):
 *     label[off + p]                              int32 mask value
 *     rho/z/rho_risk/z_risk[(off * (E-1)) + (e-1) * H*W + p]
 *   z is the sum alpha T z (not yet divided); rho_risk and z_risk bound how
 *   much rho^e and that sum move if a marginal decision flips (walk_pixel).
 * Returns 0, -1 on a zero quaternion, -2 on bad arguments.
 */
int fso_render_masks(int64_t N, const float* mean, const float* quat, const float* scale,
                     const float* opacity, const uint64_t* member, int32_t V,
                     const fso_camera* cams, int32_t E, double tau, int32_t coverage,
                     int32_t nthreads, int32_t* label, double* rho, double* z, double* rho_risk,
                     double* z_risk) {
  if (N < 0 || V < 0 || E < 2 || E > 64) return -2;
  if (nthreads < 1) nthreads = 1;
  const fso_rule rule = {FSO_ALPHA_MIN, FSO_T_MIN, FSO_EVENT_REL};
  const int objects = E - 1;
  fso_proj* P = (fso_proj*)malloc(sizeof(fso_proj) * (size_t)(N > 0 ? N : 1));
  render_job* jobs = (render_job*)calloc((size_t)nthreads, sizeof(render_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  int status = 0;
  int64_t off = 0;
  for (int32_t v = 0; v < V && !status; ++v) {
    const fso_camera* cam = &cams[v];
    const int64_t npix = (int64_t)cam->width * cam->height;
    status = project_all(N, mean, quat, scale, opacity, cam, nthreads, 0, coverage, P);
    if (status) break;
    for (int e = 1; e <= objects; ++e) {
      view_index vi;
      index_view(N, cam, P, 1, NULL, member, 1ull << e, &vi);
      int64_t max_cand = 0;
      const int64_t nb = (int64_t)vi.bins_x * vi.bins_y;
      for (int64_t b = 0; b < nb; ++b) {
        const int64_t c = vi.bin_start[b + 1] - vi.bin_start[b];
        if (c > max_cand) max_cand = c;
      }
      const int64_t plane = off * objects + (int64_t)(e - 1) * npix;
      for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (render_job){P, &vi, cam, coverage, &rule, nthreads, t,
                               rho + plane, z + plane, rho_risk + plane, z_risk + plane,
                               (fso_hit*)malloc(sizeof(fso_hit) * (size_t)(max_cand > 0 ? max_cand : 1))};
        pthread_create(&th[t], NULL, render_worker, &jobs[t]);
      }
      for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        free(jobs[t].hits);
      }
      free_view(&vi);
    }
    /* quantisation at tau, then the smallest depth among the objects that pass */
    for (int64_t p = 0; p < npix; ++p) {
      int32_t best = 0;
      double best_d = INFINITY;
      for (int e = 1; e <= objects; ++e) {
        const int64_t k = off * objects + (int64_t)(e - 1) * npix + p;
        if (!(rho[k] > tau)) continue;
        const double d = z[k] / rho[k];
        if (d < best_d) { best_d = d; best = e; }
      }
      label[off + p] = best;
    }
    off += npix;
  }
  free(jobs);
  free(th);
  free(P);
  return status;
}
