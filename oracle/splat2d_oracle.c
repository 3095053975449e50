/*
 * splat2d_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of the 2D Gaussian surfel (2DGS) image
 * formation model that Flash-Mono's mapping backend renders and refines
 * (Sec. 3 "Preliminaries", Eq. 1; the surfel primitive of 2D Gaussian
 * Splatting, cited there), and of its analytic gradient.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may call it.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * What is computed (readings of the paper, in the paper's notation):
 *   surfel i: center mu_i, colour c_i, opacity sigma_i, rotation r_i (a
 *   quaternion, normalised here), two tangent scales s_i (Sec. 3).
 *   Camera frame: mu_c = R mu + t; tangent vectors U = s_u R t_u,
 *   V = s_v R t_v with (t_u, t_v, n) the columns of R(r); n_c = R n, turned
 *   to face the camera.  The ray through pixel x meets the surfel plane at
 *   local coordinates (u, v): with M = K [U | V | mu_c], (u, v, 1) is
 *   proportional to M^-1 x, evaluated here as adj(M) x.
 *   G = max(exp(-(u^2+v^2)/2), exp(-|x - c|^2 / (2 sigma_lp^2))) with c the
 *   projected center (object/screen low-pass max), alpha = min(alpha_max,
 *   sigma G); pairs with alpha < alpha_min are skipped; front-to-back in
 *   (depth key, index) order, w_i = alpha_i T_i with T_i = prod_{j<i}(1 -
 *   alpha_j), and the pixel stops before the first surfel that would take
 *   T below t_min.  Outputs (Eq. 1): I = sum c_i w_i + T_final bg,
 *   D = sum z_i w_i (z_i = depth of mu_c along the optical axis), A = 1 -
 *   T_final, and a camera-frame normal N = sum n_c,i w_i.  Optionally
 *   (depth_ray) z_i is taken per pixel as the depth of the ray-splat
 *   intersection point, where the object-space term decides (2DGS geometry).
 *   For a fronto-parallel surfel this is exactly Eq. 1 with the screen-space
 *   covariance Sigma = (f/z)^2 R2 diag(s^2) R2^T.
 *
 * Two decisions are taken in FP32 (the precision of the library it checks),
 * so that both sides agree bit for bit: the depth sort key
 *   z32 = fmaf(R22, mu_z, fmaf(R21, mu_y, fmaf(R20, mu_x, t_z)))
 * and nothing else.  All other arithmetic is FP64.  Decisions that FP32 and
 * FP64 could take differently (alpha near alpha_min, T near t_min, a pixel-
 * rect edge within rounding of a pixel center, the near-plane cull) are not
 * hidden: they are reported as flags so a test can exclude exactly those
 * pixels or surfels and count them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NREC 20
/* record layout (FP64): A = adj(M) row-major (9), projected center (2),
 * depth z, camera normal (3), opacity, rgb (3), det(M). */
enum { R_A = 0, R_CX = 9, R_CY = 10, R_Z = 11, R_N = 12, R_OP = 15, R_RGB = 16, R_DET = 19 };

/* surfel status */
enum { ST_VISIBLE = 0, ST_OPACITY = 1, ST_NEAR = 2, ST_EMPTY = 3, ST_INVALID = 4 };
/* surfel flags */
enum {
  SF_TILE_AMBIG = 1u,  /* tile rect or emptiness could differ under rounding */
  SF_NEAR_AMBIG = 2u,  /* near-plane cull could differ under rounding */
  SF_PIX_AMBIG = 4u    /* some pixel-rect edge is within rounding of a pixel center */
};
/* pixel flags */
enum {
  PF_ALPHA_MIN = 1u,   /* an alpha within margin of alpha_min before the stop */
  PF_T_MIN = 2u,       /* the stop decision within margin of t_min */
  PF_RECT = 4u,        /* an ambiguous rect edge decides whether a pair counts */
  PF_NEAR = 8u,        /* a near-ambiguous surfel reaches alpha_min here */
  PF_ALPHA_MAX = 16u,  /* sigma*G within margin of alpha_max (gradient only) */
  PF_BRANCH = 32u      /* object vs low-pass term tied (gradient only) */
};

typedef struct {
  int W, H;
  double fx, fy, cx, cy;
  double R[9], t[3];
  float Rf[9], tf[3];
} cam_t;

typedef struct {
  double alpha_min, alpha_max, t_min, sigma_lp, z_near, bg[3];
  int tile_w, tile_h;
  double eps_alpha, eps_t, eps_px, eps_z;
  int depth_ray;  /* depth output: 0 = z_i of the center, 1 = depth of the ray-splat intersection */
  /* Which pixel rect decides whether a pair counts in binned mode: 0 = the
   * rect of the extent (the definition), 1 = the widest and 2 = the
   * narrowest rect that rounding of the extent could give.  Variants 1 and 2
   * state the two outcomes of a rect edge within rounding of a pixel center,
   * so that a result taken at lower precision can be checked against either
   * side of that decision instead of being dropped. */
  int rect_variant;
} cfg_t;

/* cam: W, H, fx, fy, cx, cy, then the 3x4 world-to-camera matrix row-major. */
static void load_cam(const double* c, cam_t* k) {
  k->W = (int)c[0];
  k->H = (int)c[1];
  k->fx = c[2]; k->fy = c[3]; k->cx = c[4]; k->cy = c[5];
  for (int r = 0; r < 3; r++) {
    for (int j = 0; j < 3; j++) {
      k->R[r * 3 + j] = c[6 + r * 4 + j];
      k->Rf[r * 3 + j] = (float)c[6 + r * 4 + j];
    }
    k->t[r] = c[6 + r * 4 + 3];
    k->tf[r] = (float)c[6 + r * 4 + 3];
  }
}

/* cfg: alpha_min, alpha_max, t_min, sigma_lp, z_near, bg[3], tile_w, tile_h,
 * eps_alpha, eps_t, eps_px, eps_z, depth_ray, rect_variant. */
static void load_cfg(const double* c, cfg_t* k) {
  k->alpha_min = c[0]; k->alpha_max = c[1]; k->t_min = c[2];
  k->sigma_lp = c[3]; k->z_near = c[4];
  k->bg[0] = c[5]; k->bg[1] = c[6]; k->bg[2] = c[7];
  k->tile_w = (int)c[8]; k->tile_h = (int)c[9];
  k->eps_alpha = c[10]; k->eps_t = c[11]; k->eps_px = c[12]; k->eps_z = c[13];
  k->depth_ray = c[14] != 0.0;
  k->rect_variant = (int)c[15];
}

/* Rotation matrix of a unit quaternion (w, x, y, z), row-major. */
static void quat_to_rot(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* d quat_to_rot / d q: DR[e][c] = dR_e / dq_c (entry e row-major, c = w,x,y,z). */
static void quat_to_rot_jac(const double q[4], double DR[9][4]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double t[9][4] = {
      {0, 0, -4 * y, -4 * z},        {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x},
      {2 * z, 2 * y, 2 * x, 2 * w},  {0, -4 * x, 0, -4 * z},         {-2 * x, -2 * w, 2 * z, 2 * y},
      {-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y},  {0, -4 * x, -4 * y, 0}};
  memcpy(DR, t, sizeof(t));
}

/* Adjugate (transpose of the cofactor matrix) of a 3x3 matrix:
 * A[i][j] = (-1)^(i+j) * det(M without row j and column i). */
static void adj3(const double M[9], double A[9]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      int r0 = (j == 0) ? 1 : 0, r1 = (j == 2) ? 1 : 2;
      int c0 = (i == 0) ? 1 : 0, c1 = (i == 2) ? 1 : 2;
      double m = M[r0 * 3 + c0] * M[r1 * 3 + c1] - M[r0 * 3 + c1] * M[r1 * 3 + c0];
      A[i * 3 + j] = ((i + j) & 1) ? -m : m;
    }
}

/* Vector-Jacobian product of adj3: dM += (dA/dM)^T dA. */
static void adj3_vjp(const double M[9], const double dA[9], double dM[9]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      int r0 = (j == 0) ? 1 : 0, r1 = (j == 2) ? 1 : 2;
      int c0 = (i == 0) ? 1 : 0, c1 = (i == 2) ? 1 : 2;
      double g = ((i + j) & 1) ? -dA[i * 3 + j] : dA[i * 3 + j];
      dM[r0 * 3 + c0] += g * M[r1 * 3 + c1];
      dM[r1 * 3 + c1] += g * M[r0 * 3 + c0];
      dM[r0 * 3 + c1] -= g * M[r1 * 3 + c0];
      dM[r1 * 3 + c0] -= g * M[r0 * 3 + c1];
    }
}

static void matvec(const double R[9], const double x[3], double y[3]) {
  for (int r = 0; r < 3; r++) y[r] = R[r * 3] * x[0] + R[r * 3 + 1] * x[1] + R[r * 3 + 2] * x[2];
}
static void matTvec(const double R[9], const double x[3], double y[3]) {
  for (int c = 0; c < 3; c++) y[c] = R[c] * x[0] + R[3 + c] * x[1] + R[6 + c] * x[2];
}
static void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Everything the forward and the chain rule need about one (view, surfel). */
typedef struct {
  double qn, qh[4], Rs[9];
  double mc[3], tu[3], tv[3], U[3], V[3], nw[3], nc[3], flip;
  double M[9], A[9];
  double su, sv;
} geom_t;

static int make_geom(const float* mu, const float* sc, const float* qq, const cam_t* c, geom_t* g) {
  double q[4] = {qq[0], qq[1], qq[2], qq[3]};
  g->qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(g->qn > 0)) return 0;
  for (int i = 0; i < 4; i++) g->qh[i] = q[i] / g->qn;
  quat_to_rot(g->qh, g->Rs);
  for (int r = 0; r < 3; r++) {
    g->tu[r] = g->Rs[r * 3 + 0];
    g->tv[r] = g->Rs[r * 3 + 1];
    g->nw[r] = g->Rs[r * 3 + 2];
  }
  double m[3] = {mu[0], mu[1], mu[2]};
  matvec(c->R, m, g->mc);
  for (int r = 0; r < 3; r++) g->mc[r] += c->t[r];
  g->su = sc[0];
  g->sv = sc[1];
  double a[3], b[3];
  matvec(c->R, g->tu, a);
  matvec(c->R, g->tv, b);
  for (int r = 0; r < 3; r++) {
    g->U[r] = g->su * a[r];
    g->V[r] = g->sv * b[r];
  }
  matvec(c->R, g->nw, g->nc);
  double d = g->nc[0] * g->mc[0] + g->nc[1] * g->mc[1] + g->nc[2] * g->mc[2];
  g->flip = (d > 0) ? -1.0 : 1.0;
  for (int r = 0; r < 3; r++) g->nc[r] *= g->flip;
  const double* X[3] = {g->U, g->V, g->mc};
  for (int k = 0; k < 3; k++) {
    g->M[0 * 3 + k] = c->fx * X[k][0] + c->cx * X[k][2];
    g->M[1 * 3 + k] = c->fy * X[k][1] + c->cy * X[k][2];
    g->M[2 * 3 + k] = X[k][2];
  }
  adj3(g->M, g->A);
  return 1;
}

static int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/*
 * Preprocess one view: per surfel, the render record, status, pixel rect and
 * tile rect (inclusive, x0 y0 x1 y1), the FP32 depth key bits and flags.
 * Extent (a reading; the paper gives none): the AABB of the projected
 * opacity-aware disk u^2+v^2 <= k^2, k^2 = 2 ln(sigma/alpha_min), from the
 * dual conic D = M diag(k^2, k^2, -1) M^T, united with the low-pass square
 * c +- sigma_lp k; pixel centers inside it are [ceil(lo-.5), floor(hi-.5)].
 * Culls: sigma < alpha_min; any point of the k-disk at depth <= z_near; no
 * pixel center in the extent.  amb[n*8] receives the widest and the
 * narrowest pixel rect that FP32 rounding of the extent could give
 * (x0 y0 x1 y1 each); they equal the pixel rect when no edge is close.
 */
int oracle_preprocess(int64_t n, const float* means, const float* scales, const float* quats,
                      const float* opacity, const float* rgb, const double* camv, const double* cfgv,
                      double* rec, int32_t* status, int32_t* pixrect, int32_t* tilerect,
                      int32_t* amb, uint32_t* zbits, uint32_t* sflags) {
  cam_t cam;
  cfg_t cfg;
  load_cam(camv, &cam);
  load_cfg(cfgv, &cfg);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; s++) {
    double* r = rec + s * NREC;
    int32_t* pr = pixrect + s * 4;
    int32_t* tr = tilerect + s * 4;
    int32_t* am = amb + s * 8;
    memset(r, 0, sizeof(double) * NREC);
    pr[0] = pr[1] = 0; pr[2] = pr[3] = -1;
    tr[0] = tr[1] = 0; tr[2] = tr[3] = -1;
    for (int k = 0; k < 8; k++) am[k] = (k & 2) ? -1 : 0;
    sflags[s] = 0;
    const float* mu = means + 3 * s;
    float z32 = fmaf(cam.Rf[8], mu[2], fmaf(cam.Rf[7], mu[1], fmaf(cam.Rf[6], mu[0], cam.tf[2])));
    memcpy(&zbits[s], &z32, 4);
    geom_t g;
    if (!make_geom(mu, scales + 2 * s, quats + 4 * s, &cam, &g)) {
      status[s] = ST_INVALID;
      continue;
    }
    double op = opacity[s];
    for (int k = 0; k < 9; k++) r[R_A + k] = g.A[k];
    r[R_CX] = g.M[2] / g.M[8];
    r[R_CY] = g.M[5] / g.M[8];
    r[R_Z] = g.mc[2];
    /* det(M), from M adj(M) = det(M) I */
    r[R_DET] = g.M[0] * g.A[0] + g.M[1] * g.A[3] + g.M[2] * g.A[6];
    for (int k = 0; k < 3; k++) r[R_N + k] = g.nc[k];
    r[R_OP] = op;
    for (int k = 0; k < 3; k++) r[R_RGB + k] = rgb[3 * s + k];

    if (op < cfg.alpha_min) {
      status[s] = ST_OPACITY;
      continue;
    }
    double k2 = 2.0 * log(op / cfg.alpha_min);
    double kk = sqrt(k2);
    double zmin = g.mc[2] - kk * sqrt(g.U[2] * g.U[2] + g.V[2] * g.V[2]);
    int near_amb = fabs(zmin - cfg.z_near) < cfg.eps_z * (1.0 + fabs(g.mc[2]));
    if (near_amb) sflags[s] |= SF_NEAR_AMBIG | SF_TILE_AMBIG;
    if (zmin <= cfg.z_near && !near_amb) {
      status[s] = ST_NEAR;
      continue;
    }
    double D[9];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        D[i * 3 + j] = k2 * (g.M[i * 3 + 0] * g.M[j * 3 + 0] + g.M[i * 3 + 1] * g.M[j * 3 + 1]) -
                       g.M[i * 3 + 2] * g.M[j * 3 + 2];
    /* tangent lines x = X: D00 - 2 X D02 + X^2 D22 = 0 (likewise y). */
    double ext[2][2];
    for (int ax = 0; ax < 2; ax++) {
      double dii = D[ax * 3 + ax], di2 = D[ax * 3 + 2], d22 = D[8];
      double disc = di2 * di2 - dii * d22;
      if (disc < 0) disc = 0;
      double r1 = (di2 + sqrt(disc)) / d22, r2 = (di2 - sqrt(disc)) / d22;
      double c0 = (ax == 0) ? r[R_CX] : r[R_CY];
      double rlp = cfg.sigma_lp * kk;
      double lo = fmin(fmin(r1, r2), c0 - rlp), hi = fmax(fmax(r1, r2), c0 + rlp);
      ext[ax][0] = lo;
      ext[ax][1] = hi;
    }
    int lim[2] = {cam.W - 1, cam.H - 1};
    int tsz[2] = {cfg.tile_w, cfg.tile_h};
    int p0[2], p1[2], p0min[2], p0max[2], p1min[2], p1max[2];
    for (int ax = 0; ax < 2; ax++) {
      double lo = ext[ax][0], hi = ext[ax][1];
      double eps = cfg.eps_px * (1.0 + (hi - lo));
      double e0 = lo - 0.5, e1 = hi - 0.5;
      int a0 = (int)ceil(e0), a1 = (int)floor(e1);
      p0[ax] = a0; p1[ax] = a1;
      p0min[ax] = p0max[ax] = a0;
      p1min[ax] = p1max[ax] = a1;
      double m0 = nearbyint(e0), m1 = nearbyint(e1);
      if (fabs(e0 - m0) < eps) { p0min[ax] = (int)m0; p0max[ax] = (int)m0 + 1; }
      if (fabs(e1 - m1) < eps) { p1min[ax] = (int)m1 - 1; p1max[ax] = (int)m1; }
      p0[ax] = iclamp(p0[ax], 0, lim[ax] + 1);
      p1[ax] = iclamp(p1[ax], -1, lim[ax]);
      p0min[ax] = iclamp(p0min[ax], 0, lim[ax] + 1);
      p0max[ax] = iclamp(p0max[ax], 0, lim[ax] + 1);
      p1min[ax] = iclamp(p1min[ax], -1, lim[ax]);
      p1max[ax] = iclamp(p1max[ax], -1, lim[ax]);
      if (p0min[ax] != p0max[ax] || p1min[ax] != p1max[ax]) sflags[s] |= SF_PIX_AMBIG;
    }
    am[0] = p0min[0]; am[1] = p0min[1]; am[2] = p1max[0]; am[3] = p1max[1];
    am[4] = p0max[0]; am[5] = p0max[1]; am[6] = p1min[0]; am[7] = p1min[1];
    int nonempty = p0[0] <= p1[0] && p0[1] <= p1[1];
    int maybe_nonempty = p0min[0] <= p1max[0] && p0min[1] <= p1max[1];
    int surely_nonempty = p0max[0] <= p1min[0] && p0max[1] <= p1min[1];
    if (maybe_nonempty != surely_nonempty) sflags[s] |= SF_TILE_AMBIG;
    for (int ax = 0; ax < 2; ax++) {
      if (p0min[ax] / tsz[ax] != p0max[ax] / tsz[ax]) sflags[s] |= SF_TILE_AMBIG;
      if (p1min[ax] >= 0 && p1min[ax] / tsz[ax] != p1max[ax] / tsz[ax]) sflags[s] |= SF_TILE_AMBIG;
    }
    if (zmin <= cfg.z_near) {
      status[s] = ST_NEAR;
      continue;
    }
    if (!nonempty) {
      status[s] = ST_EMPTY;
      continue;
    }
    status[s] = ST_VISIBLE;
    pr[0] = p0[0]; pr[1] = p0[1]; pr[2] = p1[0]; pr[3] = p1[1];
    tr[0] = p0[0] / cfg.tile_w; tr[1] = p0[1] / cfg.tile_h;
    tr[2] = p1[0] / cfg.tile_w; tr[3] = p1[1] / cfg.tile_h;
  }
  return 0;
}

/* One (pixel, surfel) evaluation in FP64. */
typedef struct {
  double alpha, raw, G, u, v, a, b, c, rho_obj, rho_lp;
  double z;   /* depth the pair contributes to the depth output */
  int obj, clamped, zray;
} eval_t;

static void eval_pair(const double* r, double px, double py, const cfg_t* cfg, eval_t* e) {
  const double* A = r + R_A;
  e->a = A[0] * px + A[1] * py + A[2];
  e->b = A[3] * px + A[4] * py + A[5];
  e->c = A[6] * px + A[7] * py + A[8];
  if (e->c != 0) {
    e->u = e->a / e->c;
    e->v = e->b / e->c;
    e->rho_obj = e->u * e->u + e->v * e->v;
  } else {
    e->u = e->v = 0;
    e->rho_obj = INFINITY;
  }
  double dx = px - r[R_CX], dy = py - r[R_CY];
  e->rho_lp = (cfg->sigma_lp > 0) ? (dx * dx + dy * dy) / (cfg->sigma_lp * cfg->sigma_lp) : INFINITY;
  e->obj = e->rho_obj <= e->rho_lp;
  double rho = e->obj ? e->rho_obj : e->rho_lp;
  e->G = exp(-0.5 * rho);
  e->raw = r[R_OP] * e->G;
  e->clamped = e->raw > cfg->alpha_max;
  e->alpha = e->clamped ? cfg->alpha_max : e->raw;
  /* Depth of the pair.  Default: the surfel center's depth z_i (Eq. 1).
   * With depth_ray, where the object-space term decides: the depth of the
   * point where the pixel's ray meets the surfel plane.  That point is
   * u U + v V + mu_c with (u, v, 1) = adj(M) x / c, and K times it equals
   * M (u, v, 1) = det(M) x / c, whose third entry is det(M) / c. */
  e->zray = cfg->depth_ray && e->obj && e->c != 0;
  e->z = e->zray ? r[R_DET] / e->c : r[R_Z];
}

/* Candidate order: ascending (z32 bits, surfel index). */
static const uint32_t* g_sort_z;
static int cmp_order(const void* pa, const void* pb) {
  int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
  uint32_t za = g_sort_z[a], zb = g_sort_z[b];
  if (za != zb) return za < zb ? -1 : 1;
  return (a > b) - (a < b);
}

/* A blended entry of one pixel, kept for the reverse pass. */
typedef struct {
  int64_t s;
  eval_t e;
  double T;
} blend_t;

typedef struct {
  int64_t n;
  const double* rec;
  const int32_t* status;
  const int32_t* pixrect;
  const int32_t* amb;
  const uint32_t* sflags;
  int64_t* order;   /* depth order of candidates */
  int64_t n_order;
  int mode;         /* 0: definition (every pixel, every surfel); 1: binned */
  /* binned mode: per tile list of candidate indices, in depth order */
  int64_t* tile_start;
  int64_t* tile_list;
  int tiles_x, tiles_y;
} view_t;

static int in_rect(const int32_t* rc, int x, int y) { return x >= rc[0] && x <= rc[2] && y >= rc[1] && y <= rc[3]; }

static void build_view(view_t* V, int mode, int64_t n, const double* rec, const int32_t* status,
                       const int32_t* pixrect, const int32_t* amb, const uint32_t* zbits,
                       const uint32_t* sflags, const cam_t* cam, const cfg_t* cfg) {
  V->n = n; V->rec = rec; V->status = status; V->pixrect = pixrect; V->amb = amb;
  V->sflags = sflags; V->mode = mode;
  V->order = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  V->n_order = 0;
  for (int64_t s = 0; s < n; s++) {
    int st = status[s];
    const int32_t* w = amb + 8 * s;
    int wide_nonempty = w[0] <= w[2] && w[1] <= w[3];
    int cand;
    if (mode == 0)
      cand = st == ST_VISIBLE || st == ST_EMPTY || ((sflags[s] & SF_NEAR_AMBIG) && st == ST_NEAR);
    else
      cand = wide_nonempty && (st == ST_VISIBLE || sflags[s] != 0);
    if (cand) V->order[V->n_order++] = s;
  }
  g_sort_z = zbits;
  qsort(V->order, (size_t)V->n_order, sizeof(int64_t), cmp_order);
  V->tile_start = NULL;
  V->tile_list = NULL;
  V->tiles_x = (cam->W + cfg->tile_w - 1) / cfg->tile_w;
  V->tiles_y = (cam->H + cfg->tile_h - 1) / cfg->tile_h;
  if (mode == 1) {
    int64_t nt = (int64_t)V->tiles_x * V->tiles_y;
    int64_t* cnt = (int64_t*)calloc((size_t)nt + 1, sizeof(int64_t));
    /* a surfel is listed in every tile its widest possible pixel rect touches */
    for (int pass = 0; pass < 2; pass++) {
      if (pass == 1) {
        V->tile_start = (int64_t*)calloc((size_t)nt + 1, sizeof(int64_t));
        for (int64_t t = 0; t < nt; t++) V->tile_start[t + 1] = V->tile_start[t] + cnt[t];
        V->tile_list = (int64_t*)malloc(sizeof(int64_t) * (V->tile_start[nt] > 0 ? V->tile_start[nt] : 1));
        memset(cnt, 0, sizeof(int64_t) * nt);
      }
      for (int64_t k = 0; k < V->n_order; k++) {
        int64_t s = V->order[k];
        const int32_t* rc = amb + 8 * s;   /* widest rect: every pixel that might count */
        for (int ty = rc[1] / cfg->tile_h; ty <= rc[3] / cfg->tile_h; ty++)
          for (int tx = rc[0] / cfg->tile_w; tx <= rc[2] / cfg->tile_w; tx++) {
            int64_t t = (int64_t)ty * V->tiles_x + tx;
            if (pass == 1) V->tile_list[V->tile_start[t] + cnt[t]] = s;
            cnt[t]++;
          }
      }
    }
    free(cnt);
  }
}

static void free_view(view_t* V) {
  free(V->order);
  free(V->tile_start);
  free(V->tile_list);
}

/*
 * Walk one pixel front to back.  Blended entries are appended to `out`
 * (capacity cap) when out != NULL.  Returns the number blended; fills the
 * outputs, T_final, flags and a hash of the decision sequence.
 */
static int64_t walk_pixel(const view_t* V, const cfg_t* cfg, int ix, int iy, double* o8, double* tfinal,
                          uint32_t* pflags, uint64_t* hash, blend_t* out, int64_t cap) {
  double px = ix + 0.5, py = iy + 0.5;
  double T = 1.0, C[3] = {0, 0, 0}, Dd = 0, N[3] = {0, 0, 0};
  uint32_t fl = 0;
  uint64_t h = 1469598103934665603ull;
  int64_t nb = 0;
  const int64_t* list;
  int64_t len;
  if (V->mode == 1) {
    int64_t t = (int64_t)(iy / cfg->tile_h) * V->tiles_x + (ix / cfg->tile_w);
    list = V->tile_list + V->tile_start[t];
    len = V->tile_start[t + 1] - V->tile_start[t];
  } else {
    list = V->order;
    len = V->n_order;
  }
  for (int64_t k = 0; k < len; k++) {
    int64_t s = list[k];
    const double* r = V->rec + s * NREC;
    int st = V->status[s];
    uint32_t sf = V->sflags[s];
    int counts;     /* does the oracle blend this pair (if alpha allows)? */
    uint32_t maybe = 0;  /* could the library decide differently? */
    if (V->mode == 1) {
      if (!in_rect(V->amb + 8 * s, ix, iy)) continue;
      counts = (st == ST_VISIBLE) && in_rect(V->pixrect + 4 * s, ix, iy);
      if (cfg->rect_variant == 1)  /* widest: the loop above already required it */
        counts = st == ST_VISIBLE || st == ST_EMPTY;
      else if (cfg->rect_variant == 2)  /* narrowest */
        counts = (st == ST_VISIBLE) && in_rect(V->amb + 8 * s + 4, ix, iy);
      if (!in_rect(V->amb + 8 * s + 4, ix, iy)) maybe |= PF_RECT;
    } else {
      counts = (st == ST_VISIBLE || st == ST_EMPTY);
    }
    if (sf & SF_NEAR_AMBIG) maybe |= PF_NEAR;
    eval_t e;
    eval_pair(r, px, py, cfg, &e);
    if (fabs(e.alpha - cfg->alpha_min) <= cfg->eps_alpha * cfg->alpha_min) fl |= PF_ALPHA_MIN;
    if (e.alpha < cfg->alpha_min) continue;
    fl |= maybe;
    if (!counts) continue;
    double Tn = T * (1.0 - e.alpha);
    if (fabs(Tn - cfg->t_min) <= cfg->eps_t * cfg->t_min) fl |= PF_T_MIN;
    if (Tn < cfg->t_min) break;
    if (fabs(e.raw - cfg->alpha_max) <= cfg->eps_alpha * cfg->alpha_max) fl |= PF_ALPHA_MAX;
    if (fabs(e.rho_obj - e.rho_lp) <= 1e-6 * (1.0 + e.rho_lp)) fl |= PF_BRANCH;
    double w = e.alpha * T;
    for (int ch = 0; ch < 3; ch++) C[ch] += w * r[R_RGB + ch];
    Dd += w * e.z;
    for (int ch = 0; ch < 3; ch++) N[ch] += w * r[R_N + ch];
    if (out && nb < cap) {
      out[nb].s = s;
      out[nb].e = e;
      out[nb].T = T;
    }
    nb++;
    h = (h ^ (uint64_t)(s * 4 + e.obj * 2 + e.clamped)) * 1099511628211ull;
    T = Tn;
  }
  if (o8) {
    for (int ch = 0; ch < 3; ch++) o8[ch] = C[ch] + T * cfg->bg[ch];
    o8[3] = Dd;
    for (int ch = 0; ch < 3; ch++) o8[4 + ch] = N[ch];
    o8[7] = 1.0 - T;
  }
  if (tfinal) *tfinal = T;
  if (pflags) *pflags = fl;
  if (hash) *hash = h ^ (uint64_t)nb;
  return nb;
}

/*
 * Render one view.  mode 0 = definition (all surfels at all pixels, the
 * authority), 1 = binned (each surfel only at pixels inside its pixel rect).
 * out: [8][H][W] planar = r, g, b, depth, nx, ny, nz, alpha.
 */
int oracle_render(int mode, int64_t n, const double* rec, const int32_t* status, const int32_t* pixrect,
                  const int32_t* amb, const uint32_t* zbits, const uint32_t* sflags, const double* camv,
                  const double* cfgv, double* out, double* tfinal, int32_t* nblend, uint32_t* pflags,
                  uint64_t* phash) {
  cam_t cam;
  cfg_t cfg;
  load_cam(camv, &cam);
  load_cfg(cfgv, &cfg);
  view_t V;
  build_view(&V, mode, n, rec, status, pixrect, amb, zbits, sflags, &cam, &cfg);
  int64_t P = (int64_t)cam.W * cam.H;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t p = 0; p < P; p++) {
    int ix = (int)(p % cam.W), iy = (int)(p / cam.W);
    double o8[8];
    double tf;
    uint32_t fl;
    uint64_t h;
    int64_t nb = walk_pixel(&V, &cfg, ix, iy, o8, &tf, &fl, &h, NULL, 0);
    for (int c = 0; c < 8; c++) out[c * P + p] = o8[c];
    tfinal[p] = tf;
    nblend[p] = (int32_t)nb;
    pflags[p] = fl;
    phash[p] = h;
  }
  free_view(&V);
  return 0;
}

/*
 * Render only the listed pixels (indices into the W*H image); outputs are
 * [8][npix].  Used to check large images on a sample of pixels.
 */
int oracle_render_pixels(int mode, int64_t n, const double* rec, const int32_t* status,
                         const int32_t* pixrect, const int32_t* amb, const uint32_t* zbits,
                         const uint32_t* sflags, const double* camv, const double* cfgv, int64_t npix,
                         const int64_t* pix, double* out, double* tfinal, int32_t* nblend,
                         uint32_t* pflags) {
  cam_t cam;
  cfg_t cfg;
  load_cam(camv, &cam);
  load_cfg(cfgv, &cfg);
  view_t V;
  build_view(&V, mode, n, rec, status, pixrect, amb, zbits, sflags, &cam, &cfg);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < npix; i++) {
    int ix = (int)(pix[i] % cam.W), iy = (int)(pix[i] / cam.W);
    double o8[8];
    double tf;
    uint32_t fl;
    uint64_t h;
    int64_t nb = walk_pixel(&V, &cfg, ix, iy, o8, &tf, &fl, &h, NULL, 0);
    for (int c = 0; c < 8; c++) out[c * npix + i] = o8[c];
    tfinal[i] = tf;
    nblend[i] = (int32_t)nb;
    pflags[i] = fl;
  }
  free_view(&V);
  return 0;
}

/*
 * The listed pixels under k configurations (cfgv: k rows of cfg values that
 * differ only in their thresholds and rect_variant; the first row's tile
 * size builds the view); out is [k][8][npix].  Used to check a pixel whose
 * decisions are within rounding against each outcome of those decisions.
 */
int oracle_render_pixels_variants(int mode, int64_t n, const double* rec, const int32_t* status,
                                  const int32_t* pixrect, const int32_t* amb, const uint32_t* zbits,
                                  const uint32_t* sflags, const double* camv, const double* cfgv, int k,
                                  int ncfg, int64_t npix, const int64_t* pix, double* out) {
  cam_t cam;
  cfg_t cfg0;
  load_cam(camv, &cam);
  load_cfg(cfgv, &cfg0);
  view_t V;
  build_view(&V, mode, n, rec, status, pixrect, amb, zbits, sflags, &cam, &cfg0);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
  for (int c = 0; c < k; c++)
    for (int64_t i = 0; i < npix; i++) {
      cfg_t cfg;
      load_cfg(cfgv + (int64_t)c * ncfg, &cfg);
      int ix = (int)(pix[i] % cam.W), iy = (int)(pix[i] / cam.W);
      double o8[8];
      walk_pixel(&V, &cfg, ix, iy, o8, NULL, NULL, NULL, NULL, 0);
      for (int ch = 0; ch < 8; ch++) out[((int64_t)c * 8 + ch) * npix + i] = o8[ch];
    }
  free_view(&V);
  return 0;
}

/*
 * Error attribution for pruning (Sec. 4.3, "Map Fusion": primitives that
 * contribute to pixels with high RGB or depth error are removed).  Reading:
 * a surfel contributes to a pixel when the pixel blends it (alpha >=
 * alpha_min, before the pixel's stop); for each surfel, max_err[s] is raised
 * to the largest err[p] over the pixels p it contributes to.  err is a
 * caller-given per-pixel error [H][W] (>= 0).  Pixels are walked one by one.
 */
int oracle_max_error(int mode, int64_t n, const double* rec, const int32_t* status, const int32_t* pixrect,
                     const int32_t* amb, const uint32_t* zbits, const uint32_t* sflags, const double* camv,
                     const double* cfgv, const double* err, double* max_err) {
  cam_t cam;
  cfg_t cfg;
  load_cam(camv, &cam);
  load_cfg(cfgv, &cfg);
  view_t V;
  build_view(&V, mode, n, rec, status, pixrect, amb, zbits, sflags, &cam, &cfg);
  int64_t cap = 4096;
  blend_t* list = (blend_t*)malloc(sizeof(blend_t) * cap);
  for (int iy = 0; iy < cam.H; iy++)
    for (int ix = 0; ix < cam.W; ix++) {
      int64_t nb = walk_pixel(&V, &cfg, ix, iy, NULL, NULL, NULL, NULL, list, cap);
      if (nb > cap) {
        cap = nb;
        list = (blend_t*)realloc(list, sizeof(blend_t) * cap);
        nb = walk_pixel(&V, &cfg, ix, iy, NULL, NULL, NULL, NULL, list, cap);
      }
      double e = err[(int64_t)iy * cam.W + ix];
      for (int64_t k = 0; k < nb; k++)
        if (e > max_err[list[k].s]) max_err[list[k].s] = e;
    }
  free(list);
  free_view(&V);
  return 0;
}

/*
 * Depth distortion of one view (the regulariser of the 2DGS surfel the paper
 * adopts, Sec. 3): per pixel, over its blended entries in blending order,
 *     D = 2 sum_i sum_{j<i} w_i w_j (z_i - z_j),
 * z the depth each entry contributes to the depth output.  When those
 * depths do not decrease along the blending order -- always for the center
 * depth, which is the sort key -- this is sum_{i,j} w_i w_j |z_i - z_j|.
 * Written as the plain double sum.  out: [H][W].
 */
int oracle_render_dist(int mode, int64_t n, const double* rec, const int32_t* status, const int32_t* pixrect,
                       const int32_t* amb, const uint32_t* zbits, const uint32_t* sflags, const double* camv,
                       const double* cfgv, double* out) {
  cam_t cam;
  cfg_t cfg;
  load_cam(camv, &cam);
  load_cfg(cfgv, &cfg);
  view_t V;
  build_view(&V, mode, n, rec, status, pixrect, amb, zbits, sflags, &cam, &cfg);
  int64_t P = (int64_t)cam.W * cam.H;
#pragma omp parallel
  {
    int64_t cap = 4096;
    blend_t* list = (blend_t*)malloc(sizeof(blend_t) * cap);
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; p++) {
      int ix = (int)(p % cam.W), iy = (int)(p / cam.W);
      int64_t nb = walk_pixel(&V, &cfg, ix, iy, NULL, NULL, NULL, NULL, list, cap);
      if (nb > cap) {
        cap = nb;
        list = (blend_t*)realloc(list, sizeof(blend_t) * cap);
        nb = walk_pixel(&V, &cfg, ix, iy, NULL, NULL, NULL, NULL, list, cap);
      }
      double d = 0;
      for (int64_t i = 0; i < nb; i++)
        for (int64_t j = 0; j < i; j++) {
          double wi = list[i].e.alpha * list[i].T, wj = list[j].e.alpha * list[j].T;
          d += 2.0 * wi * wj * (list[i].e.z - list[j].e.z);
        }
      out[p] = d;
    }
    free(list);
  }
  free_view(&V);
  return 0;
}

/*
 * Reverse pass of one view.  Upstream gradients g8 are [8][H][W] (same
 * channel order as the outputs).  Record gradients (dL/d of the 19 record
 * fields) are accumulated into grec[n*20]; the chain rule to the surfel
 * parameters and the camera se(3) tangent is oracle_chain().  Only pixels
 * whose index is listed in pix (or all pixels if npix < 0) contribute.
 * gdist ([H][W] or NULL) is the upstream gradient of the depth distortion
 * (oracle_render_dist).
 */
int oracle_render_bwd(int mode, int64_t n, const double* rec, const int32_t* status,
                      const int32_t* pixrect, const int32_t* amb, const uint32_t* zbits,
                      const uint32_t* sflags, const double* camv, const double* cfgv, const double* g8,
                      int64_t npix, const int64_t* pix, double* grec, const double* gdist) {
  cam_t cam;
  cfg_t cfg;
  load_cam(camv, &cam);
  load_cfg(cfgv, &cfg);
  view_t V;
  build_view(&V, mode, n, rec, status, pixrect, amb, zbits, sflags, &cam, &cfg);
  int64_t P = (int64_t)cam.W * cam.H;
  int64_t cnt = npix < 0 ? P : npix;
#pragma omp parallel
  {
    int64_t cap = 4096;
    blend_t* list = (blend_t*)malloc(sizeof(blend_t) * cap);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < cnt; i++) {
      int64_t p = npix < 0 ? i : pix[i];
      int ix = (int)(p % cam.W), iy = (int)(p / cam.W);
      double tf;
      int64_t nb = walk_pixel(&V, &cfg, ix, iy, NULL, &tf, NULL, NULL, list, cap);
      if (nb > cap) {
        cap = nb;
        list = (blend_t*)realloc(list, sizeof(blend_t) * cap);
        nb = walk_pixel(&V, &cfg, ix, iy, NULL, &tf, NULL, NULL, list, cap);
      }
      double dC[3], dD, dN[3], dA;
      for (int c = 0; c < 3; c++) dC[c] = g8[c * P + p];
      dD = g8[3 * P + p];
      for (int c = 0; c < 3; c++) dN[c] = g8[(4 + c) * P + p];
      dA = g8[7 * P + p];
      double px = ix + 0.5, py = iy + 0.5;
      /* suffix sums S_f = sum over later blended entries of w f, colour incl. T_final bg */
      double SC[3] = {tf * cfg.bg[0], tf * cfg.bg[1], tf * cfg.bg[2]}, SD = 0, SN[3] = {0, 0, 0};
      /* depth distortion D = 2 sum_i w_i (z_i A_{i-1} - B_{i-1}), A_{i-1} and
       * B_{i-1} the sums of w_j and w_j z_j in front of i.  Behind entry k:
       * Asuf = sum w_i, Bsuf = sum w_i z_i, Wsuf = sum w_i dD/dw_i. */
      const double gd = gdist ? gdist[p] : 0.0;
      double Dtot = 0, Asuf = 0, Bsuf = 0, Wsuf = 0;
      if (gd != 0)
        for (int64_t k = 0; k < nb; k++) Dtot += list[k].e.alpha * list[k].T * list[k].e.z;
      for (int64_t k = nb - 1; k >= 0; k--) {
        const blend_t* b = &list[k];
        const double* r = rec + b->s * NREC;
        double al = b->e.alpha, Ti = b->T, w = al * Ti, om = 1.0 - al;
        double g[NREC];
        memset(g, 0, sizeof(g));
        double da = 0;
        for (int c = 0; c < 3; c++) {
          g[R_RGB + c] = w * dC[c];
          da += dC[c] * (Ti * r[R_RGB + c] - SC[c] / om);
        }
        const double zi = b->e.z;
        double dzd = 0; /* dL/dz_k through the distortion */
        if (gd != 0) {
          const double Ap = 1.0 - Ti, Bp = Dtot - w * zi - Bsuf;  /* sums in front of k */
          const double Wk = 2.0 * (zi * Ap - Bp + Bsuf - zi * Asuf);   /* dD/dw_k */
          da += gd * (Wk * Ti - Wsuf / om);
          dzd = gd * 2.0 * w * (Ap - Asuf);                            /* dD/dz_k */
          Asuf += w;
          Bsuf += w * zi;
          Wsuf += Wk * w;
        }
        if (b->e.zray) {
          /* z = det(M) / c with c = A[6] px + A[7] py + A[8] */
          double dz = w * dD + dzd, c = b->e.c;
          g[R_DET] = dz / c;
          double x[3] = {px, py, 1.0};
          for (int j = 0; j < 3; j++) g[R_A + 6 + j] -= dz * zi / c * x[j];
        } else {
          g[R_Z] = w * dD + dzd;
        }
        da += dD * (Ti * zi - SD / om);
        for (int c = 0; c < 3; c++) {
          g[R_N + c] = w * dN[c];
          da += dN[c] * (Ti * r[R_N + c] - SN[c] / om);
        }
        da += dA * tf / om;
        for (int c = 0; c < 3; c++) SC[c] += w * r[R_RGB + c];
        SD += w * zi;
        for (int c = 0; c < 3; c++) SN[c] += w * r[R_N + c];
        if (!b->e.clamped) {
          g[R_OP] = da * b->e.G;
          double dG = da * r[R_OP];
          double drho = -0.5 * b->e.G * dG;
          if (b->e.obj) {
            double du = 2 * b->e.u * drho, dv = 2 * b->e.v * drho;
            double c = b->e.c;
            double dac = du / c, dbc = dv / c, dcc = -(b->e.u * du + b->e.v * dv) / c;
            double x[3] = {px, py, 1.0};
            for (int j = 0; j < 3; j++) {
              g[R_A + 0 + j] = dac * x[j];
              g[R_A + 3 + j] = dbc * x[j];
              g[R_A + 6 + j] += dcc * x[j];
            }
          } else {
            double s2 = cfg.sigma_lp * cfg.sigma_lp;
            g[R_CX] = drho * (-2.0 * (px - r[R_CX]) / s2);
            g[R_CY] = drho * (-2.0 * (py - r[R_CY]) / s2);
          }
        }
        double* gr = grec + b->s * NREC;
        for (int f = 0; f < NREC; f++) {
          if (g[f] != 0) {
#pragma omp atomic
            gr[f] += g[f];
          }
        }
      }
    }
    free(list);
  }
  free_view(&V);
  return 0;
}

/*
 * Chain rule from record gradients to surfel parameters and to the camera
 * pose, for one view.  Parameter gradients are accumulated (+=) into
 * g_means[n*3], g_scales[n*2], g_quats[n*4], g_opacity[n], g_rgb[n*3];
 * g_pose[6] += (d rho, d phi) for the left perturbation T_cw <- Exp(xi) T_cw,
 * xi = (rho, phi), at xi = 0.
 */
int oracle_chain(int64_t n, const float* means, const float* scales, const float* quats,
                 const int32_t* status, const double* camv, const double* grec, double* g_means,
                 double* g_scales, double* g_quats, double* g_opacity, double* g_rgb, double* g_pose) {
  cam_t cam;
  load_cam(camv, &cam);
  double pose[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t s = 0; s < n; s++) {
    if (status[s] != ST_VISIBLE) continue;
    const double* gr = grec + s * NREC;
    int nz = 0;
    for (int f = 0; f < NREC; f++) nz |= gr[f] != 0;
    if (!nz) continue;
    geom_t g;
    if (!make_geom(means + 3 * s, scales + 2 * s, quats + 4 * s, &cam, &g)) continue;
    double dM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    adj3_vjp(g.M, gr + R_A, dM);
    /* d det(M) / d M_ij = adj(M)_ji */
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) dM[i * 3 + j] += gr[R_DET] * g.A[j * 3 + i];
    double m22 = g.M[8];
    dM[2] += gr[R_CX] / m22;
    dM[5] += gr[R_CY] / m22;
    dM[8] -= (gr[R_CX] * g.M[2] + gr[R_CY] * g.M[5]) / (m22 * m22);
    double dX[3][3];
    for (int k = 0; k < 3; k++) {
      dX[k][0] = cam.fx * dM[0 * 3 + k];
      dX[k][1] = cam.fy * dM[1 * 3 + k];
      dX[k][2] = cam.cx * dM[0 * 3 + k] + cam.cy * dM[1 * 3 + k] + dM[2 * 3 + k];
    }
    double *dU = dX[0], *dV = dX[1], *dmc = dX[2];
    dmc[2] += gr[R_Z];
    const double* dnc = gr + R_N;
    /* pose: d mu_c / d rho = I, d X / d phi = -[X]x for X in {mu_c, U, V, n_c} */
    double cr[3];
    for (int k = 0; k < 3; k++) pose[k] += dmc[k];
    cross(g.mc, dmc, cr); for (int k = 0; k < 3; k++) pose[3 + k] += cr[k];
    cross(g.U, dU, cr); for (int k = 0; k < 3; k++) pose[3 + k] += cr[k];
    cross(g.V, dV, cr); for (int k = 0; k < 3; k++) pose[3 + k] += cr[k];
    cross(g.nc, dnc, cr); for (int k = 0; k < 3; k++) pose[3 + k] += cr[k];
    /* back to world */
    double dmu[3], wU[3], wV[3], wn[3];
    matTvec(cam.R, dmc, dmu);
    matTvec(cam.R, dU, wU);
    matTvec(cam.R, dV, wV);
    matTvec(cam.R, dnc, wn);
    double dsu = 0, dsv = 0;
    for (int k = 0; k < 3; k++) {
      dsu += g.tu[k] * wU[k];
      dsv += g.tv[k] * wV[k];
    }
    double dRs[9];
    for (int k = 0; k < 3; k++) {
      dRs[k * 3 + 0] = g.su * wU[k];
      dRs[k * 3 + 1] = g.sv * wV[k];
      dRs[k * 3 + 2] = g.flip * wn[k];
    }
    double DR[9][4];
    quat_to_rot_jac(g.qh, DR);
    double dqh[4] = {0, 0, 0, 0};
    for (int e = 0; e < 9; e++)
      for (int c = 0; c < 4; c++) dqh[c] += DR[e][c] * dRs[e];
    double dot = 0;
    for (int c = 0; c < 4; c++) dot += g.qh[c] * dqh[c];
    for (int k = 0; k < 3; k++) g_means[3 * s + k] += dmu[k];
    g_scales[2 * s + 0] += dsu;
    g_scales[2 * s + 1] += dsv;
    for (int c = 0; c < 4; c++) g_quats[4 * s + c] += (dqh[c] - g.qh[c] * dot) / g.qn;
    g_opacity[s] += gr[R_OP];
    for (int c = 0; c < 3; c++) g_rgb[3 * s + c] += gr[R_RGB + c];
  }
  for (int k = 0; k < 6; k++) g_pose[k] += pose[k];
  return 0;
}

/*
 * Tile binning and sort, stated plainly: every visible (view, surfel) pair
 * emits one instance per tile of its tile rect, in (view, surfel) order,
 * with key = (tile_base[view] + ty*tiles_x[view] + tx) << 32 | z32 bits and
 * value = global surfel index; the instances are then stably sorted by key.
 * Records are concatenated over views (view v owns count[v] records).
 * Returns the instance count (written only if <= cap).
 */
typedef struct {
  uint64_t key;
  int64_t seq;
  uint32_t val;
} inst_t;

static int cmp_inst(const void* pa, const void* pb) {
  const inst_t* a = (const inst_t*)pa;
  const inst_t* b = (const inst_t*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return (a->seq > b->seq) - (a->seq < b->seq);
}

int64_t oracle_bin_sort(int n_views, const int64_t* count, const int32_t* status, const int32_t* tilerect,
                        const uint32_t* zbits, const int64_t* surfel_index, const int64_t* tile_base,
                        const int32_t* tiles_x, uint64_t* keys, uint32_t* vals, int64_t cap) {
  int64_t total = 0, rbase = 0;
  for (int v = 0; v < n_views; v++) {
    for (int64_t i = 0; i < count[v]; i++) {
      int64_t r = rbase + i;
      if (status[r] != ST_VISIBLE) continue;
      const int32_t* tr = tilerect + 4 * r;
      total += (int64_t)(tr[2] - tr[0] + 1) * (tr[3] - tr[1] + 1);
    }
    rbase += count[v];
  }
  if (total > cap) return total;
  inst_t* buf = (inst_t*)malloc(sizeof(inst_t) * (total > 0 ? total : 1));
  int64_t k = 0;
  rbase = 0;
  for (int v = 0; v < n_views; v++) {
    for (int64_t i = 0; i < count[v]; i++) {
      int64_t r = rbase + i;
      if (status[r] != ST_VISIBLE) continue;
      const int32_t* tr = tilerect + 4 * r;
      for (int ty = tr[1]; ty <= tr[3]; ty++)
        for (int tx = tr[0]; tx <= tr[2]; tx++) {
          uint64_t tile = (uint64_t)(tile_base[v] + (int64_t)ty * tiles_x[v] + tx);
          buf[k].key = (tile << 32) | zbits[r];
          buf[k].seq = k;
          buf[k].val = (uint32_t)surfel_index[r];
          k++;
        }
    }
    rbase += count[v];
  }
  qsort(buf, (size_t)total, sizeof(inst_t), cmp_inst);
  for (int64_t i = 0; i < total; i++) {
    keys[i] = buf[i].key;
    vals[i] = buf[i].val;
  }
  free(buf);
  return total;
}
