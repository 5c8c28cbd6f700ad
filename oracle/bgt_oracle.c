/*
 * bgt_oracle.c -- plain, slow FP64 CPU oracle of the BG-Triangle
 * differentiable rasterizer (Wu, Dai, Yao, Tuytelaars, Yu: "BG-Triangle:
 * Bezier Gaussian Triangle for 3D Vectorization and Rendering", CVPR 2025).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file. The CUDA library never links
 * it, and the two share no code, header, table or constant.
 *
 * Stages and the passage each follows:
 *   bgto_bernstein / bgto_decasteljau  Sec. 3.1, Eq. 1-2 (and the textbook
 *                                      de Casteljau recursion, a cross-check)
 *   bgto_raster     Sec. 3.2 "Tessellation and Rasterization": tessellate
 *                   every primitive into flat triangles, rasterize with a
 *                   depth test, interpolate barycentrics -> I_id, I_uv.
 *   prepare()       boundary set B (same paragraph), boundary points and
 *                   their radius sigma (Sec. 3.2, "Discontinuity-Aware Alpha
 *                   Blending", first paragraph), sub-primitive Gaussians
 *                   (Eq. 3 position, Eq. 4 colour, Eq. 5 at attribute-map
 *                   resolution 1, EWA projection as in 3DGS).
 *   w_coef()        Eq. 6 with gamma of Eq. 7; the candidate boundary point
 *                   is the one with the smallest gamma among the boundary
 *                   points of the Gaussian's own primitive (Sec. 3.2
 *                   "Rendering Acceleration").
 *   bgto_render     Eq. 8 and point-based front-to-back alpha blending
 *                   C = sum T_i alpha_i c_i + T_n c_bg (supplementary,
 *                   "Backward Derivative", blending equations).
 *   bgto_backward   supplementary "Backward Derivative": dl/dc_i, dl/dalpha_i,
 *                   dl/dw, dl/db, gamma', dl/dp_ijk = dl/dS_q B_ijk; the
 *                   projection / EWA factors the paper leaves to 3DGS are
 *                   derived here by the chain rule.
 *
 * Precision: FP64 throughout, except where floating point decides an
 * integer inside the rasterizer (which flat triangle covers a pixel and which
 * one wins the depth test). Those decisions are taken in FP32 with one fixed
 * sequence of correctly rounded operations, the same one the CUDA kernel
 * uses, so that I_id and B are reproducible bit for bit. Vertex positions are
 * snapped to a 1/256-pixel grid and coverage uses exact 64-bit edge functions.
 * Build with -ffp-contract=off so that no multiply-add is fused implicitly.
 *
 * Readings where the paper is silent (each is a named constant or argument):
 *   control-point order i = n..0, j = n-i..0, k = n-i-j; u<->i, v<->j, w<->k.
 *   tessellation: uniform level-L lattice (a/L, b/L), L^2 flat triangles.
 *   fill rule: pixel centre at integer (x, y); covered if every edge function
 *   is > 0, or == 0 on an edge with dy < 0 || (dy == 0 && dx > 0).
 *   depth ties: smaller (primitive, sub-triangle) id wins.
 *   B: foreground pixels with a 4-neighbour (inside the image) whose id differs.
 *   sigma_b = k_b * fx * r_b / z_b (projected radius of the isotropic boundary
 *   Gaussian, k_b standard deviations).
 *   w: gamma* = min over boundary points b of primitive g of gamma(|q-b|;
 *   sigma_b), 1 if g has none; w = gamma* if I_id(q) == g else 1 - gamma*.
 *   alpha = min(alpha_max, o w G); pairs with alpha < alpha_min are dropped;
 *   blending stops before the pair that would take T below t_stop.
 *   survivors are composited in (depth, Gaussian index) order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXN 4
#define MAXCP 15

/* instability flags, per pixel */
#define F_AMIN 1
#define F_AMAX 2
#define F_TSTOP 4
#define F_DEPTH 8
#define F_SAT 16
#define F_ARGMIN 32
#define F_DZERO 64 /* |q - b*| below tol_d: direction of dl/db ill-conditioned */
#define F_DEPTHG 128 /* depth near-tie of equal-colour neighbours: C unchanged, gradient attribution not */

/* record widths of the optional stage outputs */
#define GREC 14 /* pix, prim, mux, muy, Ka, Kb, Kc, depth, r, g, b, o, rx, ry */
#define BREC 6  /* pix, prim, bx, by, sigma, z */

static int ncp(int n) { return (n + 1) * (n + 2) / 2; }

static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; i++) r *= i;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1-2: Bernstein basis, control points in the i-descending order       */
/* ------------------------------------------------------------------------ */

static void bernstein(int n, double u, double v, double w, double *B) {
  int idx = 0;
  for (int i = n; i >= 0; i--)
    for (int j = n - i; j >= 0; j--) {
      int k = n - i - j;
      B[idx++] = fact(n) / (fact(i) * fact(j) * fact(k)) * pow(u, i) * pow(v, j) * pow(w, k);
    }
}

int bgto_bernstein(int n, double u, double v, double w, double *B) {
  if (n < 0 || n > MAXN) return -1;
  bernstein(n, u, v, w, B);
  return 0;
}

/* de Casteljau recursion on the triangular net: each level replaces the net
 * of degree r by u P_{i+1,j,k} + v P_{i,j+1,k} + w P_{i,j,k+1} of degree r-1. */
int bgto_decasteljau(int n, const double *ctrl, double u, double v, double w, double *out) {
  if (n < 0 || n > MAXN) return -1;
  double net[MAXCP][3], nxt[MAXCP][3];
  for (int a = 0; a < ncp(n); a++)
    for (int c = 0; c < 3; c++) net[a][c] = ctrl[3 * a + c];
  for (int r = n; r >= 1; r--) {
    int m = r - 1;
    for (int i = m; i >= 0; i--)
      for (int j = m - i; j >= 0; j--) {
        int k = m - i - j;
        int dst = (m - i) * (m - i + 1) / 2 + k;
        int pi = (r - (i + 1)) * (r - (i + 1) + 1) / 2 + k;  /* (i+1, j, k) at degree r */
        int pj = (r - i) * (r - i + 1) / 2 + k;              /* (i, j+1, k) */
        int pk = (r - i) * (r - i + 1) / 2 + (k + 1);        /* (i, j, k+1) */
        for (int c = 0; c < 3; c++) nxt[dst][c] = u * net[pi][c] + v * net[pj][c] + w * net[pk][c];
      }
    memcpy(net, nxt, sizeof(net));
  }
  for (int c = 0; c < 3; c++) out[c] = net[0][c];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Rasterizer: the integer decisions in FP32, fixed operation order         */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t X, Y; /* snapped screen position, 1/256 px */
  float Z;      /* camera-space depth */
  float iz;     /* 1 / Z */
  int valid;
} fvert;

static float coef_f(int n, int i, int j, int k) {
  return (float)(fact(n) / (fact(i) * fact(j) * fact(k)));
}

/* One lattice vertex (a/L, b/L) of primitive `cp` in FP32: Bernstein sum with
 * fused multiply-adds in control-point order, world->camera, pinhole
 * projection, snap to 1/256 px. Every operation is one IEEE rounding. */
static fvert vertex_f32(int n, const float *cp, int a, int b, int L, const float *cam,
                        float near_z) {
  fvert o;
  float u = (float)a / (float)L;
  float v = (float)b / (float)L;
  float w = (float)(L - a - b) / (float)L;
  float pu[MAXN + 1], pv[MAXN + 1], pw[MAXN + 1];
  pu[0] = pv[0] = pw[0] = 1.0f;
  for (int m = 1; m <= n; m++) {
    pu[m] = pu[m - 1] * u;
    pv[m] = pv[m - 1] * v;
    pw[m] = pw[m - 1] * w;
  }
  float Sx = 0.0f, Sy = 0.0f, Sz = 0.0f;
  int idx = 0;
  for (int i = n; i >= 0; i--)
    for (int j = n - i; j >= 0; j--) {
      int k = n - i - j;
      float B = ((coef_f(n, i, j, k) * pu[i]) * pv[j]) * pw[k];
      Sx = fmaf(B, cp[3 * idx + 0], Sx);
      Sy = fmaf(B, cp[3 * idx + 1], Sy);
      Sz = fmaf(B, cp[3 * idx + 2], Sz);
      idx++;
    }
  const float *R = cam, *t = cam + 9;
  float Xc = R[0] * Sx; Xc = fmaf(R[1], Sy, Xc); Xc = fmaf(R[2], Sz, Xc); Xc = Xc + t[0];
  float Yc = R[3] * Sx; Yc = fmaf(R[4], Sy, Yc); Yc = fmaf(R[5], Sz, Yc); Yc = Yc + t[1];
  float Zc = R[6] * Sx; Zc = fmaf(R[7], Sy, Zc); Zc = fmaf(R[8], Sz, Zc); Zc = Zc + t[2];
  o.valid = (Zc >= near_z);
  o.Z = Zc;
  o.iz = 1.0f / Zc;
  float xs = Xc * o.iz, ys = Yc * o.iz;
  float x = fmaf(cam[12], xs, cam[14]);
  float y = fmaf(cam[13], ys, cam[15]);
  if (!(fabsf(x) <= 1048576.0f && fabsf(y) <= 1048576.0f)) o.valid = 0;
  if (o.valid) {
    o.X = (int32_t)rintf(x * 256.0f);
    o.Y = (int32_t)rintf(y * 256.0f);
  } else {
    o.X = o.Y = 0;
  }
  return o;
}

static int64_t floor_div256(int64_t a) { return (a >= 0) ? a / 256 : -((-a + 255) / 256); }
static int64_t ceil_div256(int64_t a) { return -floor_div256(-a); }

static int64_t edge_fn(const fvert *a, const fvert *b, int64_t Px, int64_t Py) {
  return (int64_t)(b->X - a->X) * (Py - a->Y) - (int64_t)(b->Y - a->Y) * (Px - a->X);
}

static int owns_zero_edge(const fvert *a, const fvert *b) {
  int32_t dx = b->X - a->X, dy = b->Y - a->Y;
  return (dy < 0) || (dy == 0 && dx > 0);
}

static uint32_t fbits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* sub-triangle s of the level-L lattice: s = 2 (a L + b) + down */
static void subtri_verts(int L, int s, int *va, int *vb) {
  int down = s & 1, cell = s >> 1;
  int a = cell / L, b = cell % L;
  if (!down) {
    va[0] = a; vb[0] = b; va[1] = a + 1; vb[1] = b; va[2] = a; vb[2] = b + 1;
  } else {
    va[0] = a + 1; vb[0] = b; va[1] = a + 1; vb[1] = b + 1; va[2] = a; vb[2] = b + 1;
  }
}

static int subtri_exists(int L, int s) {
  int down = s & 1, cell = s >> 1;
  int a = cell / L, b = cell % L;
  return down ? (a + b <= L - 2) : (a + b <= L - 1);
}

/* Rasterize every flat triangle of every primitive with a z-buffer of
 * 64-bit keys (complement of the float bits of the interpolated 1/z << 32 |
 * sub-triangle id): 1/z is affine in screen space, so at a covered pixel it is
 * sum(e_i / z_i) / area2 with the exact edge functions e_i; the nearest surface
 * has the largest 1/z and, complemented, the smallest key.
 * out_key receives the winning key per pixel (~0 for background); out_id the
 * primitive (-1 background); out_uv the perspective-correct (u, v) in FP64
 * from the exact edge functions of the winning triangle. If `ztest` is 0,
 * only out_cover (number of covering flat triangles per pixel) is filled. */
int bgto_raster(int n, int M, const float *ctrl, int L, const float *cam, int W, int H,
                float near_z, int ztest, int32_t *out_id, double *out_uv, uint64_t *out_key,
                int32_t *out_cover) {
  if (n < 1 || n > MAXN || L < 1 || W < 0 || H < 0 || M < 0) return -1;
  const int m = ncp(n);
  const int nsub = 2 * L * L;
  const int64_t P = (int64_t)W * H;
  uint64_t *zb = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
  for (int64_t p = 0; p < P; p++) zb[p] = ~(uint64_t)0;
  if (out_cover)
    for (int64_t p = 0; p < P; p++) out_cover[p] = 0;
  fvert *vt = (fvert *)malloc(sizeof(fvert) * (L + 1) * (L + 1));
  for (int g = 0; g < M; g++) {
    const float *cp = ctrl + (size_t)g * m * 3;
    for (int a = 0; a <= L; a++)
      for (int b = 0; a + b <= L; b++) vt[a * (L + 1) + b] = vertex_f32(n, cp, a, b, L, cam, near_z);
    for (int s = 0; s < nsub; s++) {
      if (!subtri_exists(L, s)) continue;
      int va[3], vb[3];
      subtri_verts(L, s, va, vb);
      fvert v0 = vt[va[0] * (L + 1) + vb[0]], v1 = vt[va[1] * (L + 1) + vb[1]],
            v2 = vt[va[2] * (L + 1) + vb[2]];
      if (!(v0.valid && v1.valid && v2.valid)) continue;
      int64_t area2 = edge_fn(&v0, &v1, v2.X, v2.Y);
      if (area2 == 0) continue;
      if (area2 < 0) {
        fvert tmp = v1; v1 = v2; v2 = tmp;
        area2 = -area2;
      }
      int64_t xmin = v0.X, xmax = v0.X, ymin = v0.Y, ymax = v0.Y;
      if (v1.X < xmin) xmin = v1.X; if (v1.X > xmax) xmax = v1.X;
      if (v2.X < xmin) xmin = v2.X; if (v2.X > xmax) xmax = v2.X;
      if (v1.Y < ymin) ymin = v1.Y; if (v1.Y > ymax) ymax = v1.Y;
      if (v2.Y < ymin) ymin = v2.Y; if (v2.Y > ymax) ymax = v2.Y;
      int64_t px0 = ceil_div256(xmin), px1 = floor_div256(xmax);
      int64_t py0 = ceil_div256(ymin), py1 = floor_div256(ymax);
      if (px0 < 0) px0 = 0; if (py0 < 0) py0 = 0;
      if (px1 > W - 1) px1 = W - 1; if (py1 > H - 1) py1 = H - 1;
      uint32_t gid = (uint32_t)g * (uint32_t)nsub + (uint32_t)s;
      for (int64_t py = py0; py <= py1; py++)
        for (int64_t px = px0; px <= px1; px++) {
          int64_t Px = px * 256, Py = py * 256;
          int64_t e0 = edge_fn(&v1, &v2, Px, Py);
          int64_t e1 = edge_fn(&v2, &v0, Px, Py);
          int64_t e2 = edge_fn(&v0, &v1, Px, Py);
          int in0 = e0 > 0 || (e0 == 0 && owns_zero_edge(&v1, &v2));
          int in1 = e1 > 0 || (e1 == 0 && owns_zero_edge(&v2, &v0));
          int in2 = e2 > 0 || (e2 == 0 && owns_zero_edge(&v0, &v1));
          if (!(in0 && in1 && in2)) continue;
          int64_t p = py * W + px;
          if (out_cover) out_cover[p]++;
          if (!ztest) continue;
          float af = (float)area2;
          float sd = (float)e0 * v0.iz;
          sd = fmaf((float)e1, v1.iz, sd);
          sd = fmaf((float)e2, v2.iz, sd);
          float inv_z = sd / af;
          uint64_t key = ((uint64_t)(~fbits(inv_z)) << 32) | gid;
          if (key < zb[p]) zb[p] = key;
        }
    }
  }
  /* resolve: primitive id and FP64 perspective-correct barycentrics */
  for (int64_t p = 0; p < P; p++) {
    if (out_key) out_key[p] = zb[p];
    if (!ztest || zb[p] == ~(uint64_t)0) {
      if (out_id) out_id[p] = -1;
      if (out_uv) { out_uv[2 * p] = 0.0; out_uv[2 * p + 1] = 0.0; }
      continue;
    }
    uint32_t gid = (uint32_t)(zb[p] & 0xffffffffu);
    int g = (int)(gid / (uint32_t)nsub), s = (int)(gid % (uint32_t)nsub);
    const float *cp = ctrl + (size_t)g * m * 3;
    int va[3], vb[3];
    subtri_verts(L, s, va, vb);
    fvert v[3];
    int ua[3], ub[3];
    for (int c = 0; c < 3; c++) {
      v[c] = vertex_f32(n, cp, va[c], vb[c], L, cam, near_z);
      ua[c] = va[c];
      ub[c] = vb[c];
    }
    int64_t area2 = edge_fn(&v[0], &v[1], v[2].X, v[2].Y);
    if (area2 < 0) {
      fvert tmp = v[1]; v[1] = v[2]; v[2] = tmp;
      int t1 = ua[1]; ua[1] = ua[2]; ua[2] = t1;
      t1 = ub[1]; ub[1] = ub[2]; ub[2] = t1;
      area2 = -area2;
    }
    int64_t Px = (p % W) * 256, Py = (p / W) * 256;
    int64_t e[3];
    e[0] = edge_fn(&v[1], &v[2], Px, Py);
    e[1] = edge_fn(&v[2], &v[0], Px, Py);
    e[2] = edge_fn(&v[0], &v[1], Px, Py);
    double wsum = 0.0, wk[3];
    for (int c = 0; c < 3; c++) {
      wk[c] = ((double)e[c] / (double)area2) / (double)v[c].Z;
      wsum += wk[c];
    }
    double u = 0.0, vv = 0.0;
    for (int c = 0; c < 3; c++) {
      u += wk[c] / wsum * ((double)ua[c] / L);
      vv += wk[c] / wsum * ((double)ub[c] / L);
    }
    if (out_id) out_id[p] = g;
    if (out_uv) { out_uv[2 * p] = u; out_uv[2 * p + 1] = vv; }
  }
  free(vt);
  free(zb);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sub-primitives and boundary points (FP64)                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  double R[9], t[3], fx, fy, cx, cy;
  int W, H;
} dcam;

typedef struct {
  int pix, prim, qx, qy;
  double u, v;
  double t[3];     /* camera-space position of S_q */
  double mu[2];    /* projected mean */
  double cov[3];   /* 2D covariance A, B, C */
  double K[3];     /* conic a, b, c (inverse covariance) */
  double col[3], o, depth;
  double Sig3[9];  /* 3D covariance */
  double quat[4], lscale[3];  /* attributes interpolated from the maps (Eq. 5) */
  double S[3];     /* world position S_q (kept for the SH direction) */
  int tex[3];      /* attribute-map texels of the interpolation and their weights */
  double tw[3];
  double rx, ry;   /* support box half extents (< 0: empty support) */
} ogauss;

typedef struct {
  int pix, prim, qx, qy;
  double u, v;
  double t[3];
  double b[2], sigma;
} obnd;

typedef struct {
  double k_b, alpha_min, alpha_max, t_stop, dilation;
  int use_boundary, all_pairs;
  double tol_alpha, tol_T, tol_z, tol_rho, tol_d;
  int attr_res;  /* leg resolution R of the rotation / scaling attribute maps */
  int sh_deg;    /* D, degree of the view-dependent SH colour (0: none) */
} oparams;

typedef struct {
  int n, M;
  const double *ctrl, *color, *opacity, *r_b, *log_scale, *quat, *bg;
  const double *sh;  /* [M][K][3] SH coefficients of bands 1..D per primitive, K = (D+1)^2 - 1 */
} oscene;

typedef struct {
  int F, Nb;
  ogauss *G;
  obnd *Bp;
  int32_t *bptr, *bidx;  /* boundary points of each primitive (CSR, bidx order) */
  int64_t *pptr;         /* candidate Gaussians of each pixel (CSR, index order) */
  int32_t *pidx;
} oprep;

static void cam_from_f32(const float *c, int W, int H, dcam *d) {
  for (int i = 0; i < 9; i++) d->R[i] = c[i];
  for (int i = 0; i < 3; i++) d->t[i] = c[9 + i];
  d->fx = c[12]; d->fy = c[13]; d->cx = c[14]; d->cy = c[15];
  d->W = W; d->H = H;
}

static void params_from(const double *p, oparams *o) {
  o->k_b = p[0]; o->alpha_min = p[1]; o->alpha_max = p[2]; o->t_stop = p[3];
  o->dilation = p[4]; o->use_boundary = (int)p[5]; o->all_pairs = (int)p[6];
  o->tol_alpha = p[7]; o->tol_T = p[8]; o->tol_z = p[9]; o->tol_rho = p[10];
  o->tol_d = p[11];
  o->attr_res = (int)p[12];
  o->sh_deg = (int)p[13];
}

/* Eq. 3 / Eq. 4: sum over control points with Bernstein weights at (u, v). */
static void interp(int n, const double *cp, double u, double v, double *out) {
  double B[MAXCP];
  bernstein(n, u, v, 1.0 - u - v, B);
  out[0] = out[1] = out[2] = 0.0;
  for (int a = 0; a < ncp(n); a++)
    for (int c = 0; c < 3; c++) out[c] += B[a] * cp[3 * a + c];
}

static void to_camera(const dcam *c, const double *S, double *t) {
  for (int r = 0; r < 3; r++) t[r] = c->R[3 * r] * S[0] + c->R[3 * r + 1] * S[1] + c->R[3 * r + 2] * S[2] + c->t[r];
}

/* 3DGS rotation of a (w, x, y, z) quaternion, normalised first. */
static void quat_rot(const double *q, double *R) {
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double r = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - r * z);     R[2] = 2 * (x * z + r * y);
  R[3] = 2 * (x * y + r * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - r * x);
  R[6] = 2 * (x * z - r * y);     R[7] = 2 * (y * z + r * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Sigma3D = (Rq S)(Rq S)^T with S = diag(exp(log_scale)). */
static void cov3d(const double *quat, const double *log_scale, double *Sig) {
  double R[9], Mx[9];
  quat_rot(quat, R);
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) Mx[3 * r + c] = R[3 * r + c] * exp(log_scale[c]);
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) {
      double s = 0;
      for (int k = 0; k < 3; k++) s += Mx[3 * r + k] * Mx[3 * c + k];
      Sig[3 * r + c] = s;
    }
}

/* Attribute maps (Eq. 5): per primitive a triangular grid of texels at the
 * nodes (i, j), i + j <= R - 1, of the level-(R - 1) barycentric lattice,
 * node (i, j) at (u, v) = (i, j) / (R - 1), stored in the control-point order
 * (i = R-1..0, then j = R-1-i..0). Theta(M, (u, v)) interpolates linearly on
 * the lattice triangle holding (u, v) (the triangle analogue of bilinear
 * texture filtering); R = 1 is one texel per primitive. */
static int tex_count(int R) { return R * (R + 1) / 2; }

static int tex_index(int R, int i, int j) {
  int n = R - 1;
  return (n - i) * (n - i + 1) / 2 + (n - i - j);
}

static void attr_weights(int R, double u, double v, int *idx, double *w) {
  int n = R - 1;
  if (n <= 0) {
    idx[0] = idx[1] = idx[2] = 0;
    w[0] = 1.0; w[1] = w[2] = 0.0;
    return;
  }
  double x = u * n, y = v * n;
  int a = (int)floor(x), b = (int)floor(y);
  if (a < 0) a = 0;
  if (b < 0) b = 0;
  if (a > n - 1) a = n - 1;
  if (b > n - 1) b = n - 1;
  if (a + b > n - 1) a = n - 1 - b;
  double fx = x - a, fy = y - b;
  if (fx + fy <= 1.0) {
    idx[0] = tex_index(R, a, b);     w[0] = 1.0 - fx - fy;
    idx[1] = tex_index(R, a + 1, b); w[1] = fx;
    idx[2] = tex_index(R, a, b + 1); w[2] = fy;
  } else {
    idx[0] = tex_index(R, a + 1, b + 1); w[0] = fx + fy - 1.0;
    idx[1] = tex_index(R, a + 1, b);     w[1] = 1.0 - fy;
    idx[2] = tex_index(R, a, b + 1);     w[2] = 1.0 - fx;
  }
}

int bgto_attr_weights(int R, double u, double v, int32_t *idx, double *w) {
  if (R < 1 || R > 16) return -1;
  int ii[3];
  attr_weights(R, u, v, ii, w);
  for (int k = 0; k < 3; k++) idx[k] = ii[k];
  return 0;
}

/* d R(q/|q|) / d q contracted with dR (3x3): dl/dq for the raw quaternion */
static void quat_rot_grad(const double *q, const double *dR, double *dq) {
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double r = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
  double g[4];
  g[0] = 2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  g[1] = 2 * (-2 * x * dR[4] + y * dR[1] + z * dR[2] + y * dR[3] - r * dR[5] + z * dR[6] + r * dR[7] - 2 * x * dR[8]);
  g[2] = 2 * (-2 * y * dR[0] + x * dR[1] + r * dR[2] + x * dR[3] + z * dR[5] - r * dR[6] + z * dR[7] - 2 * y * dR[8]);
  g[3] = 2 * (-2 * z * dR[0] - r * dR[1] + x * dR[2] + r * dR[3] - 2 * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
  /* through the normalisation: (I - qh qh^T) g / |q| */
  double qh[4] = {r, x, y, z}, d = 0;
  for (int k = 0; k < 4; k++) d += qh[k] * g[k];
  for (int k = 0; k < 4; k++) dq[k] = (g[k] - qh[k] * d) / nq;
}

/* Real spherical harmonics of bands 1..D at the unit direction d, from their
 * definition: Y_l^0 = K_l^0 P_l^0(cos t), Y_l^m = sqrt(2) K_l^m cos(m p) P_l^m(cos t),
 * Y_l^-m = sqrt(2) K_l^m sin(m p) P_l^m(cos t) (m > 0), K_l^m =
 * sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^m the associated Legendre functions
 * with the Condon-Shortley phase (three-term recurrence), t the polar angle
 * from +z and p = atan2(y, x). Y[k] for k = l^2 - 1 + (m + l), m = -l..l. */
static double factorial_d(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; i++) f *= i;
  return f;
}

static double assoc_legendre(int l, int m, double x) {
  double pmm = 1.0, somx2 = sqrt(fmax(0.0, 1.0 - x * x));
  for (int i = 1; i <= m; i++) pmm *= -(2.0 * i - 1.0) * somx2;
  if (l == m) return pmm;
  double pmm1 = x * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pmm1;
  double pll = 0.0;
  for (int ll = m + 2; ll <= l; ll++) {
    pll = ((2.0 * ll - 1.0) * x * pmm1 - (ll + m - 1.0) * pmm) / (ll - m);
    pmm = pmm1;
    pmm1 = pll;
  }
  return pll;
}

static void sh_basis(int D, const double *dir, double *Y) {
  const double PI = 3.14159265358979323846;
  double nd = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  double x = dir[0] / nd, y = dir[1] / nd, z = dir[2] / nd;
  double ph = atan2(y, x);
  for (int l = 1; l <= D; l++)
    for (int m = -l; m <= l; m++) {
      int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * PI) * factorial_d(l - am) / factorial_d(l + am));
      double P = assoc_legendre(l, am, z), val;
      if (m == 0) val = K * P;
      else if (m > 0) val = sqrt(2.0) * K * cos(am * ph) * P;
      else val = sqrt(2.0) * K * sin(am * ph) * P;
      Y[l * l - 1 + (m + l)] = val;
    }
}

int bgto_sh_basis(int D, const double *dir, double *Y) {
  if (D < 0 || D > 3) return -1;
  sh_basis(D, dir, Y);
  return 0;
}

/* camera centre in world coordinates, C = -R^T t */
static void cam_centre(const dcam *c, double *C) {
  for (int k = 0; k < 3; k++) C[k] = -(c->R[k] * c->t[0] + c->R[3 + k] * c->t[1] + c->R[6 + k] * c->t[2]);
}

/* Jacobian of the pinhole projection at camera point t, 2x3 row-major. */
static void proj_jac(const dcam *c, const double *t, double *J) {
  double tz = t[2];
  J[0] = c->fx / tz; J[1] = 0.0;         J[2] = -c->fx * t[0] / (tz * tz);
  J[3] = 0.0;        J[4] = c->fy / tz;  J[5] = -c->fy * t[1] / (tz * tz);
}

/* EWA: Sigma2D = (J W) Sigma3D (J W)^T + dilation I. */
static void cov2d(const dcam *c, const double *t, const double *Sig3, double dil, double *cov,
                  double *Tm) {
  double J[6];
  proj_jac(c, t, J);
  for (int r = 0; r < 2; r++)
    for (int k = 0; k < 3; k++)
      Tm[3 * r + k] = J[3 * r] * c->R[k] + J[3 * r + 1] * c->R[3 + k] + J[3 * r + 2] * c->R[6 + k];
  double TS[6];
  for (int r = 0; r < 2; r++)
    for (int k = 0; k < 3; k++)
      TS[3 * r + k] = Tm[3 * r] * Sig3[k] + Tm[3 * r + 1] * Sig3[3 + k] + Tm[3 * r + 2] * Sig3[6 + k];
  double S00 = TS[0] * Tm[0] + TS[1] * Tm[1] + TS[2] * Tm[2];
  double S01 = TS[0] * Tm[3] + TS[1] * Tm[4] + TS[2] * Tm[5];
  double S11 = TS[3] * Tm[3] + TS[4] * Tm[4] + TS[5] * Tm[5];
  cov[0] = S00 + dil;
  cov[1] = S01;
  cov[2] = S11 + dil;
}

static void prep_free(oprep *pr) {
  free(pr->G); free(pr->Bp); free(pr->bptr); free(pr->bidx); free(pr->pptr); free(pr->pidx);
  memset(pr, 0, sizeof(*pr));
}

/* Build Gaussians (one per foreground pixel, pixel order), boundary points
 * (pixel order), the per-primitive boundary lists and per-pixel candidate
 * lists. In all-pairs mode every Gaussian is a candidate of every pixel; in
 * box mode only those whose support box contains the pixel: outside the box
 * o G < alpha_min, and since w <= 1 the pair would be dropped anyway. */
/* pix_mask (nullable): only these pixels get candidate lists */
static int prepare(const oscene *sc, const dcam *c, const int32_t *id, const double *uv,
                   const oparams *pa, const int32_t *pix_mask, oprep *pr) {
  memset(pr, 0, sizeof(*pr));
  if (pa->attr_res < 1 || pa->attr_res > 16) return -2;
  if (pa->sh_deg < 0 || pa->sh_deg > 3 || (pa->sh_deg > 0 && !sc->sh)) return -3;
  const int W = c->W, H = c->H, n = sc->n, m = ncp(n);
  const int64_t P = (int64_t)W * H;
  int F = 0, Nb = 0;
  for (int64_t p = 0; p < P; p++)
    if (id[p] >= 0) F++;
  pr->G = (ogauss *)calloc(F > 0 ? F : 1, sizeof(ogauss));
  pr->Bp = (obnd *)calloc(F > 0 ? F : 1, sizeof(obnd));
  int gi = 0;
  for (int64_t p = 0; p < P; p++) {
    int g = id[p];
    if (g < 0) continue;
    if (g >= sc->M) return -2;
    int qx = (int)(p % W), qy = (int)(p / W);
    double u = uv[2 * p], v = uv[2 * p + 1];
    const double *cp = sc->ctrl + (size_t)g * m * 3;
    /* B: 4-neighbourhood inside the image, background counts as different */
    int isb = 0;
    if (qx > 0 && id[p - 1] != g) isb = 1;
    if (qx < W - 1 && id[p + 1] != g) isb = 1;
    if (qy > 0 && id[p - W] != g) isb = 1;
    if (qy < H - 1 && id[p + W] != g) isb = 1;
    double S[3];
    interp(n, cp, u, v, S);
    if (isb) {
      obnd *b = &pr->Bp[Nb++];
      b->pix = (int)p; b->prim = g; b->qx = qx; b->qy = qy; b->u = u; b->v = v;
      to_camera(c, S, b->t);
      b->b[0] = c->fx * b->t[0] / b->t[2] + c->cx;
      b->b[1] = c->fy * b->t[1] / b->t[2] + c->cy;
      b->sigma = pa->k_b * c->fx * sc->r_b[g] / b->t[2];
    }
    ogauss *G = &pr->G[gi++];
    G->pix = (int)p; G->prim = g; G->qx = qx; G->qy = qy; G->u = u; G->v = v;
    to_camera(c, S, G->t);
    G->depth = G->t[2];
    G->mu[0] = c->fx * G->t[0] / G->t[2] + c->cx;
    G->mu[1] = c->fy * G->t[1] / G->t[2] + c->cy;
    {
      const int R = pa->attr_res, nt = tex_count(R);
      attr_weights(R, u, v, G->tex, G->tw);
      for (int k = 0; k < 4; k++) G->quat[k] = 0.0;
      for (int k = 0; k < 3; k++) G->lscale[k] = 0.0;
      for (int e = 0; e < 3; e++) {
        const double *qt = sc->quat + 4 * ((size_t)g * nt + G->tex[e]);
        const double *st = sc->log_scale + 3 * ((size_t)g * nt + G->tex[e]);
        for (int k = 0; k < 4; k++) G->quat[k] += G->tw[e] * qt[k];
        for (int k = 0; k < 3; k++) G->lscale[k] += G->tw[e] * st[k];
      }
      cov3d(G->quat, G->lscale, G->Sig3);
    }
    double Tm[6];
    cov2d(c, G->t, G->Sig3, pa->dilation, G->cov, Tm);
    double det = G->cov[0] * G->cov[2] - G->cov[1] * G->cov[1];
    G->K[0] = G->cov[2] / det;
    G->K[1] = -G->cov[1] / det;
    G->K[2] = G->cov[0] / det;
    interp(n, sc->color + (size_t)g * m * 3, u, v, G->col);
    if (pa->sh_deg > 0) {
      /* view-dependent colour: diffuse (Eq. 4) plus SH bands 1..D of the
       * primitive's coefficients at the direction from the camera to S_q */
      const int K = (pa->sh_deg + 1) * (pa->sh_deg + 1) - 1;
      double C0[3], dir[3], Y[15];
      cam_centre(c, C0);
      for (int k = 0; k < 3; k++) dir[k] = S[k] - C0[k];
      sh_basis(pa->sh_deg, dir, Y);
      for (int k = 0; k < K; k++)
        for (int ch = 0; ch < 3; ch++) G->col[ch] += Y[k] * sc->sh[((size_t)g * K + k) * 3 + ch];
      for (int k = 0; k < 3; k++) G->S[k] = S[k];
    }
    G->o = sc->opacity[g];
    if (G->o > pa->alpha_min) {
      double lvl = 2.0 * log(G->o / pa->alpha_min);
      G->rx = sqrt(lvl * G->cov[0]) * (1.0 + 1e-9) + 1e-9;
      G->ry = sqrt(lvl * G->cov[2]) * (1.0 + 1e-9) + 1e-9;
    } else {
      G->rx = G->ry = -1.0;
    }
  }
  pr->F = F;
  pr->Nb = Nb;
  /* boundary points of each primitive, in boundary index order */
  pr->bptr = (int32_t *)calloc(sc->M + 1, sizeof(int32_t));
  pr->bidx = (int32_t *)malloc(sizeof(int32_t) * (Nb > 0 ? Nb : 1));
  for (int i = 0; i < Nb; i++) pr->bptr[pr->Bp[i].prim + 1]++;
  for (int g = 0; g < sc->M; g++) pr->bptr[g + 1] += pr->bptr[g];
  {
    int32_t *fill = (int32_t *)calloc(sc->M + 1, sizeof(int32_t));
    for (int i = 0; i < Nb; i++) {
      int g = pr->Bp[i].prim;
      pr->bidx[pr->bptr[g] + fill[g]++] = i;
    }
    free(fill);
  }
  /* candidate Gaussians per pixel */
  if (!pa->all_pairs) {
    pr->pptr = (int64_t *)calloc(P + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; pass++) {
      int64_t *fill = pass ? (int64_t *)calloc(P + 1, sizeof(int64_t)) : NULL;
      for (int i = 0; i < F; i++) {
        const ogauss *G = &pr->G[i];
        if (G->rx < 0) continue;
        int x0 = (int)ceil(G->mu[0] - G->rx), x1 = (int)floor(G->mu[0] + G->rx);
        int y0 = (int)ceil(G->mu[1] - G->ry), y1 = (int)floor(G->mu[1] + G->ry);
        if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0;
        if (x1 > W - 1) x1 = W - 1; if (y1 > H - 1) y1 = H - 1;
        for (int y = y0; y <= y1; y++)
          for (int x = x0; x <= x1; x++) {
            int64_t p = (int64_t)y * W + x;
            if (pix_mask && !pix_mask[p]) continue;
            if (!pass) pr->pptr[p + 1]++;
            else pr->pidx[pr->pptr[p] + fill[p]++] = i;
          }
      }
      if (!pass) {
        for (int64_t p = 0; p < P; p++) pr->pptr[p + 1] += pr->pptr[p];
        pr->pidx = (int32_t *)malloc(sizeof(int32_t) * (pr->pptr[P] > 0 ? pr->pptr[P] : 1));
      } else {
        free(fill);
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 6-7: blending coefficient                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
  double w, gamma, rho, d;
  int bstar;   /* boundary index of the most influential point, -1 if none */
  int sign;    /* +1: w = gamma (pixel inside g); -1: w = 1 - gamma */
  int flags;
} wres;

static double gamma_fn(double d, double sigma) {
  double x = pow(2.0, d / sigma - 1.0);
  return x < 1.0 ? x : 1.0;
}

static wres w_coef(const oprep *pr, const oparams *pa, int qx, int qy, int idq, int g) {
  wres r;
  r.bstar = -1; r.rho = INFINITY; r.d = 0.0; r.flags = 0;
  r.sign = (idq == g) ? 1 : -1;
  if (!pa->use_boundary) {
    r.gamma = 1.0;
    r.w = 1.0;
    return r;
  }
  double second = INFINITY;
  for (int k = pr->bptr[g]; k < pr->bptr[g + 1]; k++) {
    const obnd *b = &pr->Bp[pr->bidx[k]];
    double dx = qx - b->b[0], dy = qy - b->b[1];
    double d = sqrt(dx * dx + dy * dy);
    double rho = d / b->sigma;
    if (rho < r.rho) {
      second = r.rho;
      r.rho = rho;
      r.d = d;
      r.bstar = pr->bidx[k];
    } else if (rho < second) {
      second = rho;
    }
  }
  r.gamma = (r.bstar < 0) ? 1.0 : gamma_fn(r.d, pr->Bp[r.bstar].sigma);
  r.w = (r.sign > 0) ? r.gamma : 1.0 - r.gamma;
  if (r.bstar >= 0) {
    if (fabs(r.rho - 1.0) <= pa->tol_rho) r.flags |= F_SAT;
    if (r.rho < 1.0 && second - r.rho <= pa->tol_rho * (r.rho > 1.0 ? r.rho : 1.0)) r.flags |= F_ARGMIN;
    if (r.rho < 1.0 && r.d <= pa->tol_d) r.flags |= F_DZERO;
  }
  return r;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel evaluation: survivors in (depth, index) order                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int gi;
  double depth, alpha, G, wv, raw;
  int clamped;
  wres wr;
  double dx, dy;
} pair_t;

static int pair_cmp(const void *a, const void *b) {
  const pair_t *x = (const pair_t *)a, *y = (const pair_t *)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->gi > y->gi) - (x->gi < y->gi);
}

/* Survivors at pixel p: every candidate Gaussian with
 * alpha = min(alpha_max, o w G) >= alpha_min (Eq. 8), sorted by (depth, idx). */
static int collect(const oprep *pr, const oparams *pa, const int32_t *id, int W, int64_t p,
                   pair_t **buf, int *cap, int *flags) {
  int qx = (int)(p % W), qy = (int)(p / W), idq = id[p];
  int cnt = 0;
  int nc = pa->all_pairs ? pr->F : (int)(pr->pptr[p + 1] - pr->pptr[p]);
  for (int c = 0; c < nc; c++) {
    int gi = pa->all_pairs ? c : pr->pidx[pr->pptr[p] + c];
    const ogauss *G = &pr->G[gi];
    double dx = qx - G->mu[0], dy = qy - G->mu[1];
    double power = -0.5 * (G->K[0] * dx * dx + G->K[2] * dy * dy) - G->K[1] * dx * dy;
    double gv = exp(power);
    double og = G->o * gv;
    if (og < pa->alpha_min * (1.0 - pa->tol_alpha)) continue;  /* w <= 1: dropped */
    wres wr = w_coef(pr, pa, qx, qy, idq, G->prim);
    double raw = G->o * wr.w * gv;
    if (fabs(raw - pa->alpha_min) <= pa->tol_alpha * pa->alpha_min) *flags |= F_AMIN;
    if (fabs(raw - pa->alpha_max) <= pa->tol_alpha * pa->alpha_max) *flags |= F_AMAX;
    double alpha = raw < pa->alpha_max ? raw : pa->alpha_max;
    if (alpha < pa->alpha_min) continue;
    if (cnt == *cap) {
      *cap = *cap ? 2 * *cap : 64;
      *buf = (pair_t *)realloc(*buf, sizeof(pair_t) * (*cap));
    }
    pair_t *e = &(*buf)[cnt++];
    e->gi = gi; e->depth = G->depth; e->alpha = alpha; e->G = gv; e->wv = wr.w; e->raw = raw;
    e->clamped = raw >= pa->alpha_max;
    e->wr = wr;
    e->dx = dx; e->dy = dy;
  }
  qsort(*buf, cnt, sizeof(pair_t), pair_cmp);
  return cnt;
}

/* Survivors a (first in FP64 depth order) and b can be composited in the
 * other order by a renderer whose depth keys resolve 1/32 of an FP32 ulp
 * (then the index) only if the depths are that close and b has the smaller
 * index; the band is widened by `tol` relative for the FP32 inputs of the
 * renderer's depth. */
static int depth_swappable(const pair_t *a, const pair_t *b, double tol) {
  if (a->gi < b->gi) return 0;
  float fa = (float)a->depth;
  double ulp = (double)nextafterf(fa, INFINITY) - (double)fa;
  return (b->depth - a->depth) <= ulp / 32.0 + tol * a->depth;
}

static uint64_t mix64(uint64_t h, uint64_t x) {
  h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  return h;
}

/* Front-to-back compositing of the survivors; returns the number composited. */
static int composite(const pair_t *s, int cnt, const oprep *pr, const oparams *pa,
                     const double *bg, double *C, double *Tout, double *Ti, int *flags,
                     uint64_t *hash) {
  double T = 1.0;
  C[0] = C[1] = C[2] = 0.0;
  int k = 0;
  uint64_t h = 0x12345678ull;
  for (; k < cnt; k++) {
    const pair_t *e = &s[k];
    double test_T = T * (1.0 - e->alpha);
    if (fabs(test_T - pa->t_stop) <= pa->tol_T * pa->t_stop) *flags |= F_TSTOP;
    *flags |= e->wr.flags;
    const int stop_here = test_T < pa->t_stop;
    if (k + 1 < cnt && depth_swappable(e, &s[k + 1], pa->tol_z)) {
      /* Two adjacent survivors that FP32 depth keys may order the other way.
       * Swapping them leaves C unchanged when their colours are equal and the
       * stop does not fall between them (C is symmetric in the pair). */
      const double *c0 = pr->G[e->gi].col, *c1 = pr->G[s[k + 1].gi].col;
      const int same = fabs(c0[0] - c1[0]) <= 1e-9 && fabs(c0[1] - c1[1]) <= 1e-9 && fabs(c0[2] - c1[2]) <= 1e-9;
      const int next_stops = T * (1.0 - e->alpha) * (1.0 - s[k + 1].alpha) < pa->t_stop;
      *flags |= (same && !stop_here && !next_stops) ? F_DEPTHG : F_DEPTH;
    }
    if (stop_here) break;
    const ogauss *G = &pr->G[e->gi];
    for (int c = 0; c < 3; c++) C[c] += T * e->alpha * G->col[c];
    if (Ti) Ti[k] = T;
    T = test_T;
    h = mix64(h, (uint64_t)e->gi * 4 + (uint64_t)e->clamped * 2 + (uint64_t)(e->wr.rho < 1.0));
    h = mix64(h, (uint64_t)(int64_t)e->wr.bstar);
  }
  if (Ti) Ti[k] = T;
  for (int c = 0; c < 3; c++) C[c] += T * bg[c];
  *Tout = T;
  h = mix64(h, (uint64_t)k);
  *hash = h;
  return k;
}

static void scene_from(int n, int M, const double *ctrl, const double *color, const double *opacity,
                       const double *r_b, const double *log_scale, const double *quat,
                       const double *bg, const double *sh, oscene *s) {
  s->n = n; s->M = M; s->ctrl = ctrl; s->color = color; s->opacity = opacity; s->r_b = r_b;
  s->log_scale = log_scale; s->quat = quat; s->bg = bg; s->sh = sh;
}

/* Forward pass from given raster outputs (id, uv). pix_mask (nullable)
 * restricts which pixels are composited; the others are left untouched.
 * out_gauss / out_bnd (nullable, capacity W*H records) receive the
 * sub-primitive and boundary records; out_counts = {F, Nb}. */
int bgto_render(int n, int M, const double *ctrl, const double *color, const double *opacity,
                const double *r_b, const double *log_scale, const double *quat, const double *bg,
                const double *sh,
                const float *camf, int W, int H, const int32_t *id, const double *uv,
                const double *params, const int32_t *pix_mask, double *out_img, double *out_T,
                int32_t *out_n, int32_t *out_flags, uint64_t *out_hash, double *out_gauss,
                double *out_bnd, int32_t *out_counts) {
  if (n < 1 || n > MAXN || W < 0 || H < 0) return -1;
  oscene sc;
  scene_from(n, M, ctrl, color, opacity, r_b, log_scale, quat, bg, sh, &sc);
  dcam c;
  cam_from_f32(camf, W, H, &c);
  oparams pa;
  params_from(params, &pa);
  oprep pr;
  int rc = prepare(&sc, &c, id, uv, &pa, pix_mask, &pr);
  if (rc) { prep_free(&pr); return rc; }
  const int64_t P = (int64_t)W * H;
  uint64_t hall = 0;
#pragma omp parallel
  {
    pair_t *buf = NULL;
    int cap = 0;
    uint64_t hloc = 0;
#pragma omp for schedule(dynamic, 64)
    for (int64_t p = 0; p < P; p++) {
      if (pix_mask && !pix_mask[p]) continue;
      int flags = 0;
      int cnt = collect(&pr, &pa, id, W, p, &buf, &cap, &flags);
      double C[3], T;
      uint64_t h;
      int k = composite(buf, cnt, &pr, &pa, bg, C, &T, NULL, &flags, &h);
      for (int ch = 0; ch < 3; ch++) out_img[3 * p + ch] = C[ch];
      if (out_T) out_T[p] = T;
      if (out_n) out_n[p] = k;
      if (out_flags) out_flags[p] = flags;
      hloc ^= mix64(h, (uint64_t)p);
    }
#pragma omp atomic
    hall ^= hloc;
    free(buf);
  }
  if (out_hash) *out_hash = hall;
  if (out_counts) { out_counts[0] = pr.F; out_counts[1] = pr.Nb; }
  if (out_gauss)
    for (int i = 0; i < pr.F; i++) {
      const ogauss *G = &pr.G[i];
      double *r = out_gauss + (size_t)i * GREC;
      r[0] = G->pix; r[1] = G->prim; r[2] = G->mu[0]; r[3] = G->mu[1];
      r[4] = G->K[0]; r[5] = G->K[1]; r[6] = G->K[2]; r[7] = G->depth;
      r[8] = G->col[0]; r[9] = G->col[1]; r[10] = G->col[2]; r[11] = G->o;
      r[12] = G->rx; r[13] = G->ry;
    }
  if (out_bnd)
    for (int i = 0; i < pr.Nb; i++) {
      const obnd *b = &pr.Bp[i];
      double *r = out_bnd + (size_t)i * BREC;
      r[0] = b->pix; r[1] = b->prim; r[2] = b->b[0]; r[3] = b->b[1]; r[4] = b->sigma; r[5] = b->t[2];
    }
  prep_free(&pr);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Backward (supplementary "Backward Derivative") + chain rule to parameters */
/* ------------------------------------------------------------------------ */

#define GG 9 /* per-Gaussian gradient: dmu x,y; dK a,b,c; dcol r,g,b; do */

static void add_atomic(double *dst, double v) {
#pragma omp atomic
  *dst += v;
}

/* dl/d(parameters) for the loss l = sum_p sum_ch dLdC[p][ch] * C[p][ch] with
 * I_id, I_uv, B and every per-pixel discrete decision (survivor set, order,
 * clamp, stop, most influential boundary point) held fixed. Gradients are
 * accumulated (+=) into g_ctrl [M][Ncp][3], g_color [M][Ncp][3],
 * g_opacity [M], g_rb [M]. out_ggrad [F][9] and out_bgrad [Nb][3]
 * (nullable) receive the intermediate per-Gaussian and per-boundary-point
 * gradients. */
int bgto_backward(int n, int M, const double *ctrl, const double *color, const double *opacity,
                  const double *r_b, const double *log_scale, const double *quat, const double *bg,
                const double *sh,
                  const float *camf, int W, int H, const int32_t *id, const double *uv,
                  const double *params, const double *dLdC, double *g_ctrl, double *g_color,
                  double *g_opacity, double *g_rb, double *out_ggrad, double *out_bgrad,
                  double *g_log_scale, double *g_quat, double *g_sh) {
  if (n < 1 || n > MAXN || W < 0 || H < 0) return -1;
  oscene sc;
  scene_from(n, M, ctrl, color, opacity, r_b, log_scale, quat, bg, sh, &sc);
  dcam c;
  cam_from_f32(camf, W, H, &c);
  oparams pa;
  params_from(params, &pa);
  oprep pr;
  int rc = prepare(&sc, &c, id, uv, &pa, NULL, &pr);
  if (rc) { prep_free(&pr); return rc; }
  const int64_t P = (int64_t)W * H;
  double *gG = (double *)calloc((size_t)(pr.F > 0 ? pr.F : 1) * GG, sizeof(double));
  double *gB = (double *)calloc((size_t)(pr.Nb > 0 ? pr.Nb : 1) * 3, sizeof(double));
  const double LN2 = 0.69314718055994530942;

#pragma omp parallel
  {
    pair_t *buf = NULL;
    int cap = 0;
    double *Ti = NULL;
    int tcap = 0;
#pragma omp for schedule(dynamic, 64)
    for (int64_t p = 0; p < P; p++) {
      const double *dC = dLdC + 3 * p;
      if (dC[0] == 0.0 && dC[1] == 0.0 && dC[2] == 0.0) continue;
      int flags = 0;
      int cnt = collect(&pr, &pa, id, W, p, &buf, &cap, &flags);
      if (cnt + 1 > tcap) {
        tcap = cnt + 1;
        Ti = (double *)realloc(Ti, sizeof(double) * tcap);
      }
      double C[3], T;
      uint64_t h;
      int k = composite(buf, cnt, &pr, &pa, bg, C, &T, Ti, &flags, &h);
      /* colour behind pair i: S_i = sum_{j>i} T_j a_j c_j + T_n bg */
      double S[3] = {Ti[k] * bg[0], Ti[k] * bg[1], Ti[k] * bg[2]};
      for (int i = k - 1; i >= 0; i--) {
        const pair_t *e = &buf[i];
        const ogauss *G = &pr.G[e->gi];
        double *gg = gG + (size_t)e->gi * GG;
        double dl_da = 0.0;
        for (int ch = 0; ch < 3; ch++) {
          add_atomic(&gg[5 + ch], dC[ch] * Ti[i] * e->alpha);
          dl_da += dC[ch] * (Ti[i] * G->col[ch] - S[ch] / (1.0 - e->alpha));
        }
        for (int ch = 0; ch < 3; ch++) S[ch] += Ti[i] * e->alpha * G->col[ch];
        if (e->clamped) continue; /* alpha = alpha_max: constant */
        /* alpha = o w G */
        add_atomic(&gg[8], dl_da * e->wv * e->G);
        double dl_dw = dl_da * G->o * e->G;
        double dl_dpow = dl_da * G->o * e->wv * e->G;
        double dx = e->dx, dy = e->dy; /* d = q - mu */
        add_atomic(&gg[2], dl_dpow * (-0.5 * dx * dx));
        add_atomic(&gg[3], dl_dpow * (-dx * dy));
        add_atomic(&gg[4], dl_dpow * (-0.5 * dy * dy));
        add_atomic(&gg[0], dl_dpow * (G->K[0] * dx + G->K[1] * dy));
        add_atomic(&gg[1], dl_dpow * (G->K[1] * dx + G->K[2] * dy));
        /* Eq. 6-7: w = gamma or 1 - gamma, gamma = 2^(rho - 1), rho = |q-b|/sigma */
        const wres *wr = &e->wr;
        if (wr->bstar >= 0 && wr->rho < 1.0 && wr->d > 0.0) {
          const obnd *b = &pr.Bp[wr->bstar];
          double dl_drho = wr->sign * dl_dw * LN2 * wr->gamma;
          double qx = (double)(p % W), qy = (double)(p / W);
          double ux = (qx - b->b[0]) / wr->d, uy = (qy - b->b[1]) / wr->d;
          double *gb = gB + (size_t)wr->bstar * 3;
          add_atomic(&gb[0], dl_drho * (-ux / b->sigma));
          add_atomic(&gb[1], dl_drho * (-uy / b->sigma));
          add_atomic(&gb[2], dl_drho * (-wr->rho / b->sigma));
        }
      }
    }
    free(buf);
    free(Ti);
  }

  const int m = ncp(n);
  /* per Gaussian: (mu, K) -> camera point t -> S_q -> control points (Eq. 3) */
  for (int i = 0; i < pr.F; i++) {
    const ogauss *G = &pr.G[i];
    const double *gg = gG + (size_t)i * GG;
    int g = G->prim;
    double tx = G->t[0], ty = G->t[1], tz = G->t[2];
    /* conic -> covariance: dl/dSigma = -K dl/dK K (symmetric matrix form) */
    double K00 = G->K[0], K01 = G->K[1], K11 = G->K[2];
    double GK00 = gg[2], GK01 = 0.5 * gg[3], GK11 = gg[4];
    /* M1 = K GK */
    double a00 = K00 * GK00 + K01 * GK01, a01 = K00 * GK01 + K01 * GK11;
    double a10 = K01 * GK00 + K11 * GK01, a11 = K01 * GK01 + K11 * GK11;
    double GS00 = -(a00 * K00 + a01 * K01);
    double GS01 = -(a00 * K01 + a01 * K11);
    double GS10 = -(a10 * K00 + a11 * K01);
    double GS11 = -(a10 * K01 + a11 * K11);
    double GSs[4] = {GS00, 0.5 * (GS01 + GS10), 0.5 * (GS01 + GS10), GS11};
    /* Sigma2D = T Sig3 T^T + dil I, T = J W: dl/dT = 2 GS T Sig3 */
    double J[6], Tm[6];
    proj_jac(&c, G->t, J);
    for (int r = 0; r < 2; r++)
      for (int kk = 0; kk < 3; kk++)
        Tm[3 * r + kk] = J[3 * r] * c.R[kk] + J[3 * r + 1] * c.R[3 + kk] + J[3 * r + 2] * c.R[6 + kk];
    double TS[6];
    for (int r = 0; r < 2; r++)
      for (int kk = 0; kk < 3; kk++)
        TS[3 * r + kk] = Tm[3 * r] * G->Sig3[kk] + Tm[3 * r + 1] * G->Sig3[3 + kk] + Tm[3 * r + 2] * G->Sig3[6 + kk];
    double GT[6];
    for (int r = 0; r < 2; r++)
      for (int kk = 0; kk < 3; kk++)
        GT[3 * r + kk] = 2.0 * (GSs[2 * r] * TS[kk] + GSs[2 * r + 1] * TS[3 + kk]);
    /* attribute maps: dl/dSigma3D = T^T dl/dSigma2D T, Sigma3D = M M^T with
     * M = R(q) diag(exp(s)): dl/dM = 2 dl/dSigma3D M, then through R(q) and
     * exp to the interpolated q and s, and with the texel weights to the maps */
    if (g_log_scale || g_quat) {
      double GS3[9];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          double acc = 0.0;
          for (int r = 0; r < 2; r++)
            for (int s2 = 0; s2 < 2; s2++) acc += Tm[3 * r + a] * GSs[2 * r + s2] * Tm[3 * s2 + b];
          GS3[3 * a + b] = acc;
        }
      double Rq[9], sc3[3], Mx[9], GM[9], GR[9], gls[3], gq[4];
      quat_rot(G->quat, Rq);
      for (int k = 0; k < 3; k++) sc3[k] = exp(G->lscale[k]);
      for (int r = 0; r < 3; r++)
        for (int cc = 0; cc < 3; cc++) Mx[3 * r + cc] = Rq[3 * r + cc] * sc3[cc];
      for (int r = 0; r < 3; r++)
        for (int cc = 0; cc < 3; cc++) {
          double acc = 0.0;
          for (int k = 0; k < 3; k++) acc += (GS3[3 * r + k] + GS3[3 * k + r]) * Mx[3 * k + cc];
          GM[3 * r + cc] = acc;
        }
      for (int cc = 0; cc < 3; cc++) {
        double ds = 0.0;
        for (int r = 0; r < 3; r++) {
          GR[3 * r + cc] = GM[3 * r + cc] * sc3[cc];
          ds += GM[3 * r + cc] * Rq[3 * r + cc];
        }
        gls[cc] = ds * sc3[cc];
      }
      quat_rot_grad(G->quat, GR, gq);
      const int nt = tex_count(pa.attr_res);
      for (int e = 0; e < 3; e++) {
        const size_t t = (size_t)g * nt + G->tex[e];
        if (g_log_scale)
          for (int k = 0; k < 3; k++) g_log_scale[3 * t + k] += G->tw[e] * gls[k];
        if (g_quat)
          for (int k = 0; k < 4; k++) g_quat[4 * t + k] += G->tw[e] * gq[k];
      }
    }
    /* dl/dJ = dl/dT W^T */
    double GJ[6];
    for (int r = 0; r < 2; r++)
      for (int kk = 0; kk < 3; kk++)
        GJ[3 * r + kk] = GT[3 * r] * c.R[3 * kk] + GT[3 * r + 1] * c.R[3 * kk + 1] + GT[3 * r + 2] * c.R[3 * kk + 2];
    double fx = c.fx, fy = c.fy, tz2 = tz * tz, tz3 = tz2 * tz;
    double gt[3];
    gt[0] = GJ[2] * (-fx / tz2);
    gt[1] = GJ[5] * (-fy / tz2);
    gt[2] = GJ[0] * (-fx / tz2) + GJ[2] * (2.0 * fx * tx / tz3) + GJ[4] * (-fy / tz2) +
            GJ[5] * (2.0 * fy * ty / tz3);
    /* mean: mu = (fx tx/tz + cx, fy ty/tz + cy) */
    gt[0] += gg[0] * fx / tz;
    gt[1] += gg[1] * fy / tz;
    gt[2] += -gg[0] * fx * tx / tz2 - gg[1] * fy * ty / tz2;
    double gS[3];
    for (int kk = 0; kk < 3; kk++) gS[kk] = c.R[kk] * gt[0] + c.R[3 + kk] * gt[1] + c.R[6 + kk] * gt[2];
    if (pa.sh_deg > 0) {
      /* SH colour: dl/dk = Y(d) dl/dc; the direction d = (S_q - C) / |S_q - C|
       * moves with S_q: its basis derivative by FP64 central differences */
      const int K = (pa.sh_deg + 1) * (pa.sh_deg + 1) - 1;
      double C0[3], v0[3], Y[15], wk[15];
      cam_centre(&c, C0);
      for (int kk = 0; kk < 3; kk++) v0[kk] = G->S[kk] - C0[kk];
      sh_basis(pa.sh_deg, v0, Y);
      for (int k = 0; k < K; k++) {
        wk[k] = 0.0;
        for (int ch = 0; ch < 3; ch++) {
          const double coef = sc.sh[((size_t)g * K + k) * 3 + ch];
          wk[k] += gg[5 + ch] * coef;
          if (g_sh) g_sh[((size_t)g * K + k) * 3 + ch] += Y[k] * gg[5 + ch];
        }
      }
      const double hv = 1e-6 * sqrt(v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2]);
      for (int j = 0; j < 3; j++) {
        double vp[3] = {v0[0], v0[1], v0[2]}, vm[3] = {v0[0], v0[1], v0[2]}, Yp[15], Ym[15];
        vp[j] += hv;
        vm[j] -= hv;
        sh_basis(pa.sh_deg, vp, Yp);
        sh_basis(pa.sh_deg, vm, Ym);
        double dj = 0.0;
        for (int k = 0; k < K; k++) dj += wk[k] * (Yp[k] - Ym[k]) / (2.0 * hv);
        gS[j] += dj;
      }
    }
    double B[MAXCP];
    bernstein(n, G->u, G->v, 1.0 - G->u - G->v, B);
    for (int a = 0; a < m; a++)
      for (int ch = 0; ch < 3; ch++) {
        g_ctrl[((size_t)g * m + a) * 3 + ch] += B[a] * gS[ch];
        g_color[((size_t)g * m + a) * 3 + ch] += B[a] * gg[5 + ch];
      }
    g_opacity[g] += gg[8];
    if (out_ggrad)
      for (int q = 0; q < GG; q++) out_ggrad[(size_t)i * GG + q] = gg[q];
  }
  /* per boundary point: (b, sigma) -> t_b -> S_b -> control points; sigma -> r_b */
  for (int i = 0; i < pr.Nb; i++) {
    const obnd *b = &pr.Bp[i];
    const double *gb = gB + (size_t)i * 3;
    int g = b->prim;
    double tx = b->t[0], ty = b->t[1], tz = b->t[2];
    double gt[3];
    gt[0] = gb[0] * c.fx / tz;
    gt[1] = gb[1] * c.fy / tz;
    gt[2] = -gb[0] * c.fx * tx / (tz * tz) - gb[1] * c.fy * ty / (tz * tz) - gb[2] * b->sigma / tz;
    g_rb[g] += gb[2] * pa.k_b * c.fx / tz;
    double gS[3];
    for (int kk = 0; kk < 3; kk++) gS[kk] = c.R[kk] * gt[0] + c.R[3 + kk] * gt[1] + c.R[6 + kk] * gt[2];
    double B[MAXCP];
    bernstein(n, b->u, b->v, 1.0 - b->u - b->v, B);
    for (int a = 0; a < m; a++)
      for (int ch = 0; ch < 3; ch++) g_ctrl[((size_t)g * m + a) * 3 + ch] += B[a] * gS[ch];
    if (out_bgrad)
      for (int q = 0; q < 3; q++) out_bgrad[(size_t)i * 3 + q] = gb[q];
  }
  free(gG);
  free(gB);
  prep_free(&pr);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel lists for the binning / sort stage test                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t dbits;
  int32_t i;
} dkey;

static int dkey_cmp(const void *a, const void *b) {
  const dkey *x = (const dkey *)a, *y = (const dkey *)b;
  if (x->dbits != y->dbits) return x->dbits < y->dbits ? -1 : 1;
  return (x->i > y->i) - (x->i < y->i);
}

/* For each pixel, the Gaussians whose support o exp(-1/2 d^T K d) >= alpha_min
 * contains it (exact FP64 test on the given FP32 inputs), in (depth, index)
 * order. Gaussian i sits at pixel (qx, qy) + off. Writes CSR (out_ptr [P+1],
 * out_idx); returns the total, or -(needed) if `cap` is too small. */
int64_t bgto_pixel_lists(int W, int H, int count, const int32_t *qx, const int32_t *qy,
                         const float *off, const float *conic, const float *opac,
                         const float *depth, double alpha_min, int32_t *out_ptr,
                         int32_t *out_idx, int64_t cap) {
  const int64_t P = (int64_t)W * H;
  int64_t total = 0;
  dkey *tmp = (dkey *)malloc(sizeof(dkey) * (count > 0 ? count : 1));
  out_ptr[0] = 0;
  for (int64_t p = 0; p < P; p++) {
    int x = (int)(p % W), y = (int)(p / W);
    int c = 0;
    for (int i = 0; i < count; i++) {
      double mx = (double)qx[i] + (double)off[2 * i], my = (double)qy[i] + (double)off[2 * i + 1];
      double dx = x - mx, dy = y - my;
      double a = conic[3 * i], b = conic[3 * i + 1], cc = conic[3 * i + 2];
      double v = (double)opac[i] * exp(-0.5 * (a * dx * dx + cc * dy * dy) - b * dx * dy);
      if (v >= alpha_min) {
        tmp[c].dbits = fbits(depth[i]);
        tmp[c].i = i;
        c++;
      }
    }
    qsort(tmp, c, sizeof(dkey), dkey_cmp);
    for (int k = 0; k < c; k++) {
      if (total + k < cap) out_idx[total + k] = tmp[k].i;
    }
    total += c;
    out_ptr[p + 1] = (int32_t)(total < 0x7fffffff ? total : 0x7fffffff);
  }
  free(tmp);
  return total <= cap ? total : -total;
}

int bgto_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Eq. 7 on its own, for the pin tests. */
double bgto_gamma(double d, double sigma) { return gamma_fn(d, sigma); }

/* Eq. 6 blending coefficient w(q, g) for `count` (pixel, primitive) pairs,
 * with the same preparation as bgto_render. out_w[i] = w; out_b[i] = index
 * of the most influential boundary point (-1 if none). */
int bgto_wvalues(int n, int M, const double *ctrl, const double *color, const double *opacity,
                 const double *r_b, const double *log_scale, const double *quat, const double *bg,
                const double *sh,
                 const float *camf, int W, int H, const int32_t *id, const double *uv,
                 const double *params, int count, const int32_t *pix, const int32_t *prim,
                 double *out_w, int32_t *out_b) {
  oscene sc;
  scene_from(n, M, ctrl, color, opacity, r_b, log_scale, quat, bg, sh, &sc);
  dcam c;
  cam_from_f32(camf, W, H, &c);
  oparams pa;
  params_from(params, &pa);
  oprep pr;
  int rc = prepare(&sc, &c, id, uv, &pa, NULL, &pr);
  if (rc) { prep_free(&pr); return rc; }
  for (int i = 0; i < count; i++) {
    int p = pix[i];
    wres r = w_coef(&pr, &pa, p % W, p / W, id[p], prim[i]);
    out_w[i] = r.w;
    if (out_b) out_b[i] = r.bstar;
  }
  prep_free(&pr);
  return 0;
}
