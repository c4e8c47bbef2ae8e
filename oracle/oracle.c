/*
 * CPU oracle for the pixel-track cellular automaton (TEST INFRASTRUCTURE ONLY).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code with the CUDA path.  It is deliberately plain: every
 * stage is the definition written out, with no binning, blocking or reordering.
 *
 * What it computes (the paper's Patatrack chain, Sec. 2.2.1 and Fig. 2: hits of
 * neighbouring layers are joined two by two, a cellular automaton chains those pairs
 * when they share a hit, chains long enough to be track candidates are selected, and
 * each candidate is fitted for its parameters).  The paper prints no cut formula, constant
 * or fit equation, so the concrete predicates below are this library's readings:
 *
 *   r = sqrt(x*x + y*y)                                   (per hit, float32)
 *   doublet (i inner, o outer) on an allowed layer pair:   D0..D4
 *   link a=(h0,h1) -> b=(h1,h2):                           C1..C3
 *   fishbone (optional) = of two aligned active cells ending on one hit, one is removed
 *   ntuplet = every root->leaf path of linked cells with 3..6 hits
 *   dedup   = best-key-per-cell, then triplets sharing a hit with a >=4-hit survivor
 *   fit     = closed-form circle (Karimaki, NIM A305 (1991) 187) + straight z(s) line
 *
 * Arithmetic rule: every cut variable is computed in float32 with only correctly
 * rounded + - * / sqrt, in the parenthesised order written in the code, without FMA
 * contraction (compile with -ffp-contract=off).  The fit is float64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_HITS 6
#define ORC_MAX_CELLS (ORC_MAX_HITS - 1)
#define ORC_N_LAYERS 10
#define ORC_N_PAIRS 13
#define ORC_MAX_PAIRS 64
#define ORC_PI 3.14159265358979323846

typedef struct {
  float kmax;      /* max curvature, 1/cm */
  float z0max;     /* max |z| at r = 0 of the doublet's r-z line, cm */
  float cotmax;    /* max |dz/dr| of a doublet */
  float rz0;       /* r-z alignment tolerance, constant term (cm) */
  float rz1;       /* r-z alignment tolerance, term proportional to |z2 - z0| */
  float dca_b0;    /* max transverse DCA of a triplet circle whose first hit is on layer 0 */
  float dca_other; /* same, first hit on any other layer */
} orc_cuts;

/* Allowed (inner, outer) layer pairs: consecutive surfaces a primary track can cross.
 * Layer codes: 0..3 barrel, 4..6 +z disks, 7..9 -z disks. */
static const int PAIR_IN[ORC_N_PAIRS] = {0, 1, 2, 0, 1, 2, 4, 5, 0, 1, 2, 7, 8};
static const int PAIR_OUT[ORC_N_PAIRS] = {1, 2, 3, 4, 4, 4, 5, 6, 7, 7, 7, 8, 9};

/* ------------------------------------------------------------------ growable arrays */
typedef struct { int32_t* v; int64_t n, cap; } ivec;
typedef struct { float* v; int64_t n, cap; } fvec;

static void iv_push(ivec* a, int32_t x) {
  if (a->n == a->cap) {
    a->cap = a->cap ? 2 * a->cap : 1024;
    a->v = (int32_t*)realloc(a->v, (size_t)a->cap * sizeof(int32_t));
  }
  a->v[a->n++] = x;
}
static void fv_push(fvec* a, float x) {
  if (a->n == a->cap) {
    a->cap = a->cap ? 2 * a->cap : 1024;
    a->v = (float*)realloc(a->v, (size_t)a->cap * sizeof(float));
  }
  a->v[a->n++] = x;
}

/* --------------------------------------------------------------- near-threshold test */
/* A decision lhs <= rhs (or lhs > rhs) is near its threshold when
 * |lhs - rhs| <= 1e-6 * max(|lhs|, |rhs|). */
static int near_thr(float lhs, float rhs) {
  double l = lhs, r = rhs;
  double m = fabs(l) > fabs(r) ? fabs(l) : fabs(r);
  return fabs(l - r) <= 1e-6 * m;
}

/* Outcome bookkeeping for one candidate: pass/fail of the AND of its cuts, plus
 * whether a cut close to its threshold could decide the outcome. */
typedef struct { int fail_far; int fail_near; int pass_near; } cut_tally;

static void classify(cut_tally* v, int pass, float lhs, float rhs) {
  int nr = near_thr(lhs, rhs);
  if (pass) { if (nr) v->pass_near = 1; }
  else if (nr) v->fail_near = 1;
  else v->fail_far = 1;
}

/* ------------------------------------------------------------------------- doublets */
/* D0 dr > 0; D1 xi*xo + yi*yo > 0; D2 curvature of the circle through the beam spot
 * (origin) and both hits <= kmax; D3 |z at r=0| of the r-z line <= z0max;
 * D4 |dz| <= cotmax * dr.  Returns 1 if accepted; *near set if the outcome could
 * flip under a 1e-6 relative change of a cut variable. */
static int doublet_ok(const orc_cuts* c, float xi, float yi, float zi, float ri, float xo,
                      float yo, float zo, float ro, int* near) {
  cut_tally v = {0, 0, 0};
  float dx = xo - xi, dy = yo - yi, dr = ro - ri, dz = zo - zi;
  classify(&v, dr > 0.0f, dr, 0.0f);
  if (v.fail_far) { *near = 0; return 0; }
  float dot = (xi * xo) + (yi * yo);
  classify(&v, dot > 0.0f, dot, 0.0f);
  if (v.fail_far) { *near = 0; return 0; }
  float l3 = fabsf((zi * dr) - (ri * dz));
  float r3 = c->z0max * dr;
  classify(&v, l3 <= r3, l3, r3);
  if (v.fail_far) { *near = 0; return 0; }
  float l4 = fabsf(dz);
  float r4 = c->cotmax * dr;
  classify(&v, l4 <= r4, l4, r4);
  if (v.fail_far) { *near = 0; return 0; }
  float l2 = fabsf((xi * yo) - (yi * xo)) * 2.0f;
  float r2 = c->kmax * ((ri * ro) * sqrtf((dx * dx) + (dy * dy)));
  classify(&v, l2 <= r2, l2, r2);
  if (v.fail_far) { *near = 0; return 0; }
  *near = v.fail_near || v.pass_near;
  return !v.fail_near;
}

/* -------------------------------------------------------------------------- links */
/* Cells a=(h0,h1), b=(h1,h2).  C1 r-z alignment of the three hits; C2 curvature of the
 * circle through the three hits <= kmax; C3 transverse distance of closest approach of
 * that circle to the beam spot <= dcamax, division-free: |num| <= dcamax * den with
 * |num|/den = | |C| - R |.  *quality receives |num|/den. */
static int link_ok(const orc_cuts* c, float x0, float y0, float z0, float r0, int layer0,
                   float x1, float y1, float z1, float r1, float x2, float y2, float z2,
                   float r2, int* near, float* quality) {
  cut_tally v = {0, 0, 0};
  float lc1 = fabsf(((z1 - z0) * (r2 - r0)) - ((z2 - z0) * (r1 - r0)));
  float rc1 = (c->rz0 * (r2 - r0)) + (c->rz1 * fabsf(z2 - z0));
  classify(&v, lc1 <= rc1, lc1, rc1);
  if (v.fail_far) { *near = 0; return 0; }
  float ax = x1 - x0, ay = y1 - y0;
  float bx = x2 - x0, by = y2 - y0;
  float cx = x2 - x1, cy = y2 - y1;
  float a2 = (ax * ax) + (ay * ay);
  float b2 = (bx * bx) + (by * by);
  float cr = (ax * by) - (ay * bx);
  float lc2 = fabsf(cr) * 2.0f;
  float rc2 = c->kmax * ((sqrtf(a2) * sqrtf(b2)) * sqrtf((cx * cx) + (cy * cy)));
  classify(&v, lc2 <= rc2, lc2, rc2);
  if (v.fail_far) { *near = 0; return 0; }
  float D = cr * 2.0f;
  float ux = (by * a2) - (ay * b2);
  float uy = (ax * b2) - (bx * a2);
  float num = (((x0 * x0) + (y0 * y0)) * D) + (((x0 * ux) + (y0 * uy)) * 2.0f);
  float px = (x0 * D) + ux;
  float py = (y0 * D) + uy;
  float den = sqrtf((px * px) + (py * py)) + sqrtf((ux * ux) + (uy * uy));
  float dcamax = layer0 == 0 ? c->dca_b0 : c->dca_other;
  float lc3 = fabsf(num);
  float rc3 = dcamax * den;
  classify(&v, lc3 <= rc3, lc3, rc3);
  if (v.fail_far) { *near = 0; return 0; }
  *near = v.fail_near || v.pass_near;
  *quality = lc3 / den;
  return !v.fail_near;
}

/* ------------------------------------------------------------------------- result */
typedef struct {
  int64_t n_hits;
  float* r;
  /* cells: input hit indices, pair-major, then inner input order, then outer input order */
  ivec cell_in, cell_out;
  /* links (cell indices a -> b) and their quality, a-major */
  ivec link_a, link_b;
  fvec link_q;
  /* all root->leaf paths with >= 3 hits, in DFS discovery order */
  ivec nt_hits;  /* [T][6], -1 padded */
  ivec nt_cells; /* [T][5], -1 padded */
  ivec nt_n;     /* hits per ntuplet */
  fvec nt_q;
  /* survivors of the duplicate cleaning, canonical order (hit tuple ascending) */
  ivec sv_idx;   /* index into the ntuplet arrays */
  /* fits of the survivors (float64), 9 values each:
   * kappa, phi0, d0, cot_theta, z0, pt, chi2_circle, chi2_line, charge */
  double* fit;
  /* near-threshold decisions: kind (0 doublet, 1 link), h0, h1, h2 (-1 for doublets) */
  ivec near;
  int64_t n_doublet_tests, n_link_tests;
} orc_result;

/* ---------------------------------------------------------------------- ntuplets */
typedef struct {
  const int32_t* out_off; /* CSR of links by source cell */
  const int32_t* out_dst;
  const float* out_q;
  const int32_t* cell_in;
  const int32_t* cell_out;
  orc_result* res;
} dfs_ctx;

static void emit_path(dfs_ctx* d, const int32_t* path, int ncells, float q) {
  orc_result* R = d->res;
  int nh = ncells + 1;
  iv_push(&R->nt_hits, d->cell_in[path[0]]);
  for (int k = 0; k < ncells; ++k) iv_push(&R->nt_hits, d->cell_out[path[k]]);
  for (int k = nh; k < ORC_MAX_HITS; ++k) iv_push(&R->nt_hits, -1);
  for (int k = 0; k < ncells; ++k) iv_push(&R->nt_cells, path[k]);
  for (int k = ncells; k < ORC_MAX_CELLS; ++k) iv_push(&R->nt_cells, -1);
  iv_push(&R->nt_n, nh);
  fv_push(&R->nt_q, q);
}

/* Depth-first walk along out-links; q accumulates the link qualities inner -> outer. */
static void dfs(dfs_ctx* d, int32_t* path, int depth, float q) {
  int32_t a = path[depth - 1];
  int32_t lo = d->out_off[a], hi = d->out_off[a + 1];
  if (lo == hi) {
    if (depth >= 2) emit_path(d, path, depth, q);
    return;
  }
  for (int32_t l = lo; l < hi; ++l) {
    if (depth >= ORC_MAX_CELLS) break; /* unreachable with the layer graph above */
    path[depth] = d->out_dst[l];
    dfs(d, path, depth + 1, q + d->out_q[l]);
  }
}

/* Strict total order used for duplicate cleaning: more hits first, then smaller q,
 * then the hit tuple (signed, -1 padded) lexicographically ascending. */
static _Thread_local const orc_result* g_sort_res;
static int tuple_cmp(const int32_t* a, const int32_t* b) {
  for (int k = 0; k < ORC_MAX_HITS; ++k) {
    if (a[k] < b[k]) return -1;
    if (a[k] > b[k]) return 1;
  }
  return 0;
}
static int key_less(const orc_result* R, int32_t t, int32_t u) {
  int nt = R->nt_n.v[t], nu = R->nt_n.v[u];
  if (nt != nu) return nt > nu;
  float qt = R->nt_q.v[t], qu = R->nt_q.v[u];
  if (qt != qu) return qt < qu;
  return tuple_cmp(R->nt_hits.v + 6 * (int64_t)t, R->nt_hits.v + 6 * (int64_t)u) < 0;
}
static int canon_cmp(const void* pa, const void* pb) {
  int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
  return tuple_cmp(g_sort_res->nt_hits.v + 6 * (int64_t)a, g_sort_res->nt_hits.v + 6 * (int64_t)b);
}

/* ---------------------------------------------------------------------------- fit */
/* Circle: minimise sum_i (k r_i^2 - x_i sin(phi) + y_i cos(phi) + delta)^2, the
 * algebraic form of the circle used by Karimaki; its closed-form minimiser in terms of
 * the centred second moments gives phi, k, delta, which convert to curvature rho and
 * signed distance d of closest approach (circle centre (1/rho + d)(sin phi, -cos phi)).
 * This library reports kappa = -rho (kappa > 0: counter-clockwise seen from +z, moving
 * from the first to the last hit), phi0 = direction of motion at the closest approach,
 * d0 = d (closest-approach point d0 * (sin phi0, -cos phi0)).
 * Line: z = z0 + cot_theta * s with s the transverse arc length from the closest
 * approach, unweighted least squares. */
static void fit_one(int n, const double* x, const double* y, const double* z, double bfield,
                    double sig_rphi, double sig_z, double* out) {
  double mx = 0, my = 0, mr = 0;
  double r2[ORC_MAX_HITS];
  for (int i = 0; i < n; ++i) {
    r2[i] = x[i] * x[i] + y[i] * y[i];
    mx += x[i]; my += y[i]; mr += r2[i];
  }
  mx /= n; my /= n; mr /= n;
  double cxx = 0, cxy = 0, cyy = 0, cxr = 0, cyr = 0, crr = 0;
  for (int i = 0; i < n; ++i) {
    double dx = x[i] - mx, dy = y[i] - my, dr = r2[i] - mr;
    cxx += dx * dx; cxy += dx * dy; cyy += dy * dy;
    cxr += dx * dr; cyr += dy * dr; crr += dr * dr;
  }
  cxx /= n; cxy /= n; cyy /= n; cxr /= n; cyr /= n; crr /= n;
  double q1 = crr * cxy - cxr * cyr;
  double q2 = crr * (cxx - cyy) - cxr * cxr + cyr * cyr;
  double phi = 0.5 * atan2(2.0 * q1, q2);
  double s = sin(phi), c = cos(phi);
  /* travel direction: from the first towards the last hit */
  if (c * (x[n - 1] - x[0]) + s * (y[n - 1] - y[0]) < 0.0) {
    phi = phi > 0 ? phi - ORC_PI : phi + ORC_PI;
    s = -s; c = -c;
  }
  double k = (s * cxr - c * cyr) / crr;
  double delta = -k * mr + s * mx - c * my;
  double root = sqrt(1.0 - 4.0 * delta * k);
  double rho = 2.0 * k / root;
  double d = 2.0 * delta / (1.0 + root);
  double kappa = -rho;
  /* circle value F(P) = rho/2 |P|^2 - u (P . n) + rho d^2/2 + d, n = (sin, -cos) */
  double u = 1.0 + rho * d;
  double pcax = d * s, pcay = -d * c;
  double chi2c = 0.0;
  double sarc[ORC_MAX_HITS];
  for (int i = 0; i < n; ++i) {
    double F = 0.5 * rho * r2[i] - u * (x[i] * s - y[i] * c) + 0.5 * rho * d * d + d;
    double eps = 2.0 * F / (1.0 + sqrt(1.0 + 2.0 * rho * F));
    chi2c += (eps / sig_rphi) * (eps / sig_rphi);
    double lx = x[i] - pcax, ly = y[i] - pcay;
    double L = sqrt(lx * lx + ly * ly);
    double zz = 0.5 * fabs(rho) * L;
    double arc = zz > 1e-12 ? (zz < 1.0 ? asin(zz) / zz : (ORC_PI / 2) / zz) * L : L;
    sarc[i] = (c * lx + s * ly) >= 0.0 ? arc : -arc;
  }
  double ms = 0, mz = 0;
  for (int i = 0; i < n; ++i) { ms += sarc[i]; mz += z[i]; }
  ms /= n; mz /= n;
  double css = 0, csz = 0;
  for (int i = 0; i < n; ++i) {
    css += (sarc[i] - ms) * (sarc[i] - ms);
    csz += (sarc[i] - ms) * (z[i] - mz);
  }
  double cot = csz / css;
  double z0 = mz - cot * ms;
  double chi2l = 0.0;
  for (int i = 0; i < n; ++i) {
    double e = (z[i] - z0 - cot * sarc[i]) / sig_z;
    chi2l += e * e;
  }
  out[0] = kappa;
  out[1] = phi;
  out[2] = d;
  out[3] = cot;
  out[4] = z0;
  out[5] = 0.299792458 * bfield / (100.0 * fabs(kappa));
  out[6] = chi2c;
  out[7] = chi2l;
  out[8] = kappa > 0 ? -1.0 : (kappa < 0 ? 1.0 : 0.0);
}

/* -------------------------------------------------------------------- dedup */
/* Duplicate cleaning of T ntuplets (hits [T][6], cells [T][5], nh [T], q [T]; cell ids
 * < n_cells, hit ids < n_hits).  Step 1: an ntuplet survives iff, for every one of its
 * cells, it has the best key (more hits, then smaller q, then smaller hit tuple) among
 * all ntuplets containing that cell.  Step 2: a 3-hit survivor sharing any hit with a
 * survivor of >= 4 hits is dropped.  Writes survivor indices in canonical order (hit
 * tuple ascending) and returns their count. */
int64_t orc_dedup(int64_t T, const int32_t* hits, const int32_t* cells, const int32_t* nh,
                  const float* q, int64_t n_cells, int64_t n_hits, int32_t* out_idx) {
  orc_result view;
  memset(&view, 0, sizeof(view));
  view.nt_hits.v = (int32_t*)hits;
  view.nt_n.v = (int32_t*)nh;
  view.nt_q.v = (float*)q;
  const orc_result* R = &view;
  int32_t* best = (int32_t*)malloc((size_t)(n_cells > 0 ? n_cells : 1) * sizeof(int32_t));
  for (int64_t c = 0; c < n_cells; ++c) best[c] = -1;
  for (int64_t t = 0; t < T; ++t)
    for (int k = 0; k < nh[t] - 1; ++k) {
      int32_t c = cells[5 * t + k];
      if (best[c] < 0 || key_less(R, (int32_t)t, best[c])) best[c] = (int32_t)t;
    }
  uint8_t* alive = (uint8_t*)calloc((size_t)(T > 0 ? T : 1), 1);
  for (int64_t t = 0; t < T; ++t) {
    int ok = 1;
    for (int k = 0; k < nh[t] - 1; ++k)
      if (best[cells[5 * t + k]] != t) ok = 0;
    alive[t] = (uint8_t)ok;
  }
  free(best);
  uint8_t* used = (uint8_t*)calloc((size_t)(n_hits > 0 ? n_hits : 1), 1);
  for (int64_t t = 0; t < T; ++t)
    if (alive[t] && nh[t] >= 4)
      for (int k = 0; k < nh[t]; ++k) used[hits[6 * t + k]] = 1;
  for (int64_t t = 0; t < T; ++t)
    if (alive[t] && nh[t] == 3)
      for (int k = 0; k < 3; ++k)
        if (used[hits[6 * t + k]]) alive[t] = 0;
  free(used);
  int64_t S = 0;
  for (int64_t t = 0; t < T; ++t)
    if (alive[t]) out_idx[S++] = (int32_t)t;
  free(alive);
  /* canonical order: hit tuple ascending (the comparator's context is thread-local) */
  g_sort_res = R;
  if (S > 1) qsort(out_idx, (size_t)S, sizeof(int32_t), canon_cmp);
  g_sort_res = NULL;
  return S;
}

/* ------------------------------------------------------------------ whole chain */
/* ---------------------------------------------------------------------- fishbone */
/* Fishbone duplicate removal (optional).  The paper does not describe this step; this is
 * the library's reading of the overlap cleaning of the Patatrack chain.  A track that
 * crosses two overlapping sensors of one layer leaves two hits there, and the cells from
 * both to the same outer hit point the same way.  Active cells are those with at least
 * one outgoing link.  Two active cells i, j ending on the same hit h, with u = h - inner(i)
 * and v = h - inner(j) (float32, outer minus inner), are compared when their inner hits
 * lie on different layers or on different sensors of one layer: radii (barrel layers
 * 0..3) or |z| (disks) more than 0.1 cm apart, the stand-in for a sensor identity,
 * which the hit input does not carry.  They are aligned when u.v > 0 and
 * (u.v)^2 >= 0.99999 |u|^2 |v|^2.  Of an aligned pair on the same inner layer the shorter
 * cell loses (the longer lever arm stays); on different inner layers the longer one loses
 * (the consecutive-layer cell stays); equal lengths: the cell whose inner hit has the
 * larger input index loses.  A cell that loses to any aligned partner is removed with
 * every link from or to it.  Activity is taken from the links before the removal, so the
 * result does not depend on the order of the comparisons. */
#define ORC_FB_COS2 0.99999f
#define ORC_FB_SENSOR_GAP 0.1f

static int fb_loses_at(float hx, float hy, float hz, float ix, float iy, float iz, int li,
                       int64_t ki, float jx, float jy, float jz, int lj, int64_t kj) {
  if (li == lj) {
    /* one layer: only hits on different sensors (radius or |z| apart) are compared */
    const float si = li < 4 ? sqrtf((ix * ix) + (iy * iy)) : fabsf(iz);
    const float sj = lj < 4 ? sqrtf((jx * jx) + (jy * jy)) : fabsf(jz);
    if (!(fabsf(si - sj) > ORC_FB_SENSOR_GAP)) return 0;
  }
  const float ux = hx - ix, uy = hy - iy, uz = hz - iz;
  const float vx = hx - jx, vy = hy - jy, vz = hz - jz;
  const float dot = ((ux * vx) + (uy * vy)) + (uz * vz);
  const float nu = ((ux * ux) + (uy * uy)) + (uz * uz);
  const float nv = ((vx * vx) + (vy * vy)) + (vz * vz);
  if (!(dot > 0.0f) || !((dot * dot) >= (ORC_FB_COS2 * (nu * nv)))) return 0;
  if (nu == nv) return ki > kj;
  return li == lj ? nu < nv : nu > nv;
}

static int fb_loses(const float* x, const float* y, const float* z, const uint8_t* layer,
                    int32_t h, int32_t hi, int32_t hj) {
  return fb_loses_at(x[h], y[h], z[h], x[hi], y[hi], z[hi], layer[hi], hi, x[hj], y[hj], z[hj],
                     layer[hj], hj);
}

/* The fishbone comparison alone (for checks): does the cell from inner hit i (layer li,
 * input index ki) to outer hit h lose to the cell from inner hit j (lj, kj) to h?
 * h, i, j: float32 (x, y, z). */
int orc_fb_loses(const float* h, const float* i, int li, int64_t ki, const float* j, int lj,
                 int64_t kj) {
  return fb_loses_at(h[0], h[1], h[2], i[0], i[1], i[2], li, ki, j[0], j[1], j[2], lj, kj);
}

/* killed[c] = 1 for every removed cell (killed has C entries, zeroed by the caller). */
static void fishbone(int64_t n, const float* x, const float* y, const float* z,
                     const uint8_t* layer, int64_t C, const int32_t* cin, const int32_t* cout,
                     const int32_t* link_off, uint8_t* killed) {
  /* active cells grouped by outer hit (counting sort) */
  int32_t* cnt = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  for (int64_t c = 0; c < C; ++c)
    if (link_off[c + 1] > link_off[c]) cnt[cout[c] + 1]++;
  for (int64_t h = 0; h < n; ++h) cnt[h + 1] += cnt[h];
  int32_t* grp = (int32_t*)malloc((size_t)(cnt[n] > 0 ? cnt[n] : 1) * sizeof(int32_t));
  int32_t* fill = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  memcpy(fill, cnt, (size_t)(n + 1) * sizeof(int32_t));
  for (int64_t c = 0; c < C; ++c)
    if (link_off[c + 1] > link_off[c]) grp[fill[cout[c]]++] = (int32_t)c;
  for (int64_t h = 0; h < n; ++h)
    for (int32_t a = cnt[h]; a < cnt[h + 1]; ++a)
      for (int32_t b = cnt[h]; b < cnt[h + 1]; ++b)
        if (a != b && fb_loses(x, y, z, layer, (int32_t)h, cin[grp[a]], cin[grp[b]])) {
          killed[grp[a]] = 1;
          break;
        }
  free(cnt); free(grp); free(fill);
}

/* link_keep (optional, may be NULL): one flag per link accepted by the cuts, in the
 * order the plain run lists them (cell a major); links with flag 0 are removed before
 * the ntuplet search (the learned gate's decision, computed by the caller). */
/* The chain over the layer pairs pin[p] -> pout[p], p < n_pairs. */
static orc_result* reconstruct_pairs(int64_t n, const float* x, const float* y, const float* z,
                                     const uint8_t* layer, const orc_cuts* cuts, double bfield,
                                     int n_pairs, const int* pin, const int* pout,
                                     const uint8_t* link_keep, int64_t n_keep, int fishbone_on);
orc_result* orc_reconstruct_ex(int64_t n, const float* x, const float* y, const float* z,
                               const uint8_t* layer, const orc_cuts* cuts, double bfield,
                               int n_pairs, const int32_t* pin, const int32_t* pout,
                               const uint8_t* link_keep, int64_t n_keep, int fishbone_on);

orc_result* orc_reconstruct(int64_t n, const float* x, const float* y, const float* z,
                            const uint8_t* layer, const orc_cuts* cuts, double bfield) {
  return reconstruct_pairs(n, x, y, z, layer, cuts, bfield, ORC_N_PAIRS, PAIR_IN, PAIR_OUT,
                           NULL, 0, 0);
}

orc_result* orc_reconstruct_masked(int64_t n, const float* x, const float* y, const float* z,
                                   const uint8_t* layer, const orc_cuts* cuts, double bfield,
                                   const uint8_t* link_keep, int64_t n_keep) {
  return reconstruct_pairs(n, x, y, z, layer, cuts, bfield, ORC_N_PAIRS, PAIR_IN, PAIR_OUT,
                           link_keep, n_keep, 0);
}

/* The chain over a caller's layer-pair table (at most ORC_MAX_PAIRS distinct pairs of
 * layer codes < ORC_N_LAYERS, inner != outer); NULL for an invalid table.  A pair named
 * twice would make every cell on it twice, so a repeated pair is invalid. */
orc_result* orc_reconstruct_pairs(int64_t n, const float* x, const float* y, const float* z,
                                  const uint8_t* layer, const orc_cuts* cuts, double bfield,
                                  int n_pairs, const int32_t* pin, const int32_t* pout) {
  if (n_pairs < 1) return NULL;
  return orc_reconstruct_ex(n, x, y, z, layer, cuts, bfield, n_pairs, pin, pout, NULL, 0, 0);
}

/* The general entry: a layer-pair table (n_pairs = 0: the default table), an optional
 * link mask (as orc_reconstruct_masked) and fishbone_on (the fishbone step after the
 * links, applied to the links the mask keeps). */
orc_result* orc_reconstruct_ex(int64_t n, const float* x, const float* y, const float* z,
                               const uint8_t* layer, const orc_cuts* cuts, double bfield,
                               int n_pairs, const int32_t* pin, const int32_t* pout,
                               const uint8_t* link_keep, int64_t n_keep, int fishbone_on) {
  int ti[ORC_MAX_PAIRS], to[ORC_MAX_PAIRS];
  if (n_pairs == 0) {
    return reconstruct_pairs(n, x, y, z, layer, cuts, bfield, ORC_N_PAIRS, PAIR_IN, PAIR_OUT,
                             link_keep, n_keep, fishbone_on);
  }
  if (n_pairs < 1 || n_pairs > ORC_MAX_PAIRS) return NULL;
  for (int p = 0; p < n_pairs; ++p) {
    if (pin[p] < 0 || pin[p] >= ORC_N_LAYERS || pout[p] < 0 || pout[p] >= ORC_N_LAYERS ||
        pin[p] == pout[p])
      return NULL;
    for (int q = 0; q < p; ++q)
      if (ti[q] == pin[p] && to[q] == pout[p]) return NULL;
    ti[p] = pin[p];
    to[p] = pout[p];
  }
  return reconstruct_pairs(n, x, y, z, layer, cuts, bfield, n_pairs, ti, to, link_keep, n_keep,
                           fishbone_on);
}

static orc_result* reconstruct_pairs(int64_t n, const float* x, const float* y, const float* z,
                                     const uint8_t* layer, const orc_cuts* cuts, double bfield,
                                     int n_pairs, const int* pin, const int* pout,
                                     const uint8_t* link_keep, int64_t n_keep, int fishbone_on) {
  int64_t lidx = 0; /* index among all links accepted by the cuts */
  orc_result* R = (orc_result*)calloc(1, sizeof(orc_result));
  R->n_hits = n;
  R->r = (float*)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
  for (int64_t i = 0; i < n; ++i) R->r[i] = sqrtf((x[i] * x[i]) + (y[i] * y[i]));
  const float* r = R->r;

  /* hits of each layer, in input order */
  ivec by_layer[ORC_N_LAYERS];
  memset(by_layer, 0, sizeof(by_layer));
  for (int64_t i = 0; i < n; ++i)
    if (layer[i] < ORC_N_LAYERS) iv_push(&by_layer[layer[i]], (int32_t)i);

  /* doublets: every (inner, outer) hit pair of every allowed layer pair */
  for (int p = 0; p < n_pairs; ++p) {
    const ivec* LI = &by_layer[pin[p]];
    const ivec* LO = &by_layer[pout[p]];
    for (int64_t a = 0; a < LI->n; ++a) {
      int32_t i = LI->v[a];
      for (int64_t b = 0; b < LO->n; ++b) {
        int32_t o = LO->v[b];
        int near = 0;
        R->n_doublet_tests++;
        int ok = doublet_ok(cuts, x[i], y[i], z[i], r[i], x[o], y[o], z[o], r[o], &near);
        if (near) {
          iv_push(&R->near, 0); iv_push(&R->near, i); iv_push(&R->near, o); iv_push(&R->near, -1);
        }
        if (ok) { iv_push(&R->cell_in, i); iv_push(&R->cell_out, o); }
      }
    }
  }
  for (int l = 0; l < ORC_N_LAYERS; ++l) free(by_layer[l].v);
  const int64_t C = R->cell_in.n;

  /* cells grouped by inner hit (counting sort, stable) */
  int32_t* out_cnt = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  for (int64_t c = 0; c < C; ++c) out_cnt[R->cell_in.v[c] + 1]++;
  for (int64_t h = 0; h < n; ++h) out_cnt[h + 1] += out_cnt[h];
  int32_t* by_inner = (int32_t*)malloc((size_t)(C > 0 ? C : 1) * sizeof(int32_t));
  int32_t* fill = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  memcpy(fill, out_cnt, (size_t)(n + 1) * sizeof(int32_t));
  for (int64_t c = 0; c < C; ++c) by_inner[fill[R->cell_in.v[c]]++] = (int32_t)c;

  /* links: for every cell a, every cell b starting at a's outer hit */
  int32_t* link_off = (int32_t*)calloc((size_t)C + 1, sizeof(int32_t));
  uint8_t* has_in = (uint8_t*)calloc((size_t)(C > 0 ? C : 1), 1);
  for (int64_t a = 0; a < C; ++a) {
    int32_t h0 = R->cell_in.v[a], h1 = R->cell_out.v[a];
    for (int32_t k = out_cnt[h1]; k < out_cnt[h1 + 1]; ++k) {
      int32_t b = by_inner[k];
      int32_t h2 = R->cell_out.v[b];
      int near = 0;
      float q = 0.0f;
      R->n_link_tests++;
      int ok = link_ok(cuts, x[h0], y[h0], z[h0], r[h0], layer[h0], x[h1], y[h1], z[h1], r[h1],
                       x[h2], y[h2], z[h2], r[h2], &near, &q);
      if (near) {
        iv_push(&R->near, 1); iv_push(&R->near, h0); iv_push(&R->near, h1); iv_push(&R->near, h2);
      }
      if (ok && link_keep) ok = lidx < n_keep && link_keep[lidx++];
      if (ok) {
        iv_push(&R->link_a, (int32_t)a);
        iv_push(&R->link_b, b);
        fv_push(&R->link_q, q);
        has_in[b] = 1;
      }
    }
    link_off[a + 1] = (int32_t)R->link_a.n;
  }
  free(out_cnt); free(by_inner); free(fill);

  if (fishbone_on) {
    /* remove the fishbone's cells with every link from or to them */
    uint8_t* killed = (uint8_t*)calloc((size_t)(C > 0 ? C : 1), 1);
    fishbone(n, x, y, z, layer, C, R->cell_in.v, R->cell_out.v, link_off, killed);
    int64_t w = 0;
    memset(has_in, 0, (size_t)(C > 0 ? C : 1));
    for (int64_t a = 0; a < C; ++a) {
      const int32_t lo = link_off[a], hi = link_off[a + 1];
      link_off[a] = (int32_t)w;
      for (int32_t l = lo; l < hi; ++l) {
        const int32_t b = R->link_b.v[l];
        if (killed[a] || killed[b]) continue;
        R->link_a.v[w] = (int32_t)a;
        R->link_b.v[w] = b;
        R->link_q.v[w] = R->link_q.v[l];
        has_in[b] = 1;
        ++w;
      }
    }
    link_off[C] = (int32_t)w;
    R->link_a.n = R->link_b.n = R->link_q.n = w;
    free(killed);
  }

  /* ntuplets: every path from a root (no incoming link) to a leaf (no outgoing link) */
  dfs_ctx d = {link_off, R->link_b.v, R->link_q.v, R->cell_in.v, R->cell_out.v, R};
  int32_t path[ORC_MAX_CELLS];
  for (int64_t a = 0; a < C; ++a) {
    if (has_in[a]) continue;
    path[0] = (int32_t)a;
    dfs(&d, path, 1, 0.0f);
  }
  free(link_off); free(has_in);
  const int64_t T = R->nt_n.n;

  R->sv_idx.v = (int32_t*)malloc((size_t)(T > 0 ? T : 1) * sizeof(int32_t));
  R->sv_idx.cap = T > 0 ? T : 1;
  R->sv_idx.n = orc_dedup(T, R->nt_hits.v, R->nt_cells.v, R->nt_n.v, R->nt_q.v, C, n,
                          R->sv_idx.v);

  /* fits of the survivors */
  const int64_t S = R->sv_idx.n;
  R->fit = (double*)malloc((size_t)(S > 0 ? S : 1) * 9 * sizeof(double));
  for (int64_t s = 0; s < S; ++s) {
    int32_t t = R->sv_idx.v[s];
    int nh = R->nt_n.v[t];
    double hx[ORC_MAX_HITS], hy[ORC_MAX_HITS], hz[ORC_MAX_HITS];
    for (int k = 0; k < nh; ++k) {
      int32_t h = R->nt_hits.v[6 * t + k];
      hx[k] = x[h]; hy[k] = y[h]; hz[k] = z[h];
    }
    fit_one(nh, hx, hy, hz, bfield, 10e-4, 20e-4, R->fit + 9 * s);
  }
  return R;
}

/* Stand-alone fit of one hit list (float64), for closed-form checks. */
void orc_fit_hits(int n, const double* x, const double* y, const double* z, double bfield,
                  double* out9) {
  fit_one(n, x, y, z, bfield, 10e-4, 20e-4, out9);
}

/* Stand-alone predicates, for unit checks of single decisions. */
int orc_doublet_ok(const orc_cuts* c, const float* hi, const float* ho, int* near) {
  float ri = sqrtf((hi[0] * hi[0]) + (hi[1] * hi[1]));
  float ro = sqrtf((ho[0] * ho[0]) + (ho[1] * ho[1]));
  return doublet_ok(c, hi[0], hi[1], hi[2], ri, ho[0], ho[1], ho[2], ro, near);
}
int orc_link_ok(const orc_cuts* c, const float* h0, int layer0, const float* h1,
                const float* h2, int* near, float* q) {
  float r0 = sqrtf((h0[0] * h0[0]) + (h0[1] * h0[1]));
  float r1 = sqrtf((h1[0] * h1[0]) + (h1[1] * h1[1]));
  float r2 = sqrtf((h2[0] * h2[0]) + (h2[1] * h2[1]));
  return link_ok(c, h0[0], h0[1], h0[2], r0, layer0, h1[0], h1[1], h1[2], r1, h2[0], h2[1],
                 h2[2], r2, near, q);
}

/* ------------------------------------------------------------------- accessors */
void orc_sizes(const orc_result* R, int64_t* out) {
  out[0] = R->cell_in.n;
  out[1] = R->link_a.n;
  out[2] = R->nt_n.n;
  out[3] = R->sv_idx.n;
  out[4] = R->near.n / 4;
  out[5] = R->n_doublet_tests;
  out[6] = R->n_link_tests;
}
void orc_get_cells(const orc_result* R, int32_t* inner, int32_t* outer) {
  memcpy(inner, R->cell_in.v, (size_t)R->cell_in.n * 4);
  memcpy(outer, R->cell_out.v, (size_t)R->cell_out.n * 4);
}
void orc_get_links(const orc_result* R, int32_t* a, int32_t* b, float* q) {
  memcpy(a, R->link_a.v, (size_t)R->link_a.n * 4);
  memcpy(b, R->link_b.v, (size_t)R->link_b.n * 4);
  memcpy(q, R->link_q.v, (size_t)R->link_q.n * 4);
}
void orc_get_ntuplets(const orc_result* R, int32_t* hits, int32_t* cells, int32_t* nh, float* q) {
  memcpy(hits, R->nt_hits.v, (size_t)R->nt_hits.n * 4);
  memcpy(cells, R->nt_cells.v, (size_t)R->nt_cells.n * 4);
  memcpy(nh, R->nt_n.v, (size_t)R->nt_n.n * 4);
  memcpy(q, R->nt_q.v, (size_t)R->nt_q.n * 4);
}
void orc_get_survivors(const orc_result* R, int32_t* idx, double* fit) {
  memcpy(idx, R->sv_idx.v, (size_t)R->sv_idx.n * 4);
  memcpy(fit, R->fit, (size_t)R->sv_idx.n * 9 * sizeof(double));
}
void orc_get_near(const orc_result* R, int32_t* rec) {
  memcpy(rec, R->near.v, (size_t)R->near.n * 4);
}
void orc_get_radius(const orc_result* R, float* r) { memcpy(r, R->r, (size_t)R->n_hits * 4); }

void orc_free(orc_result* R) {
  if (!R) return;
  free(R->r);
  free(R->cell_in.v); free(R->cell_out.v);
  free(R->link_a.v); free(R->link_b.v); free(R->link_q.v);
  free(R->nt_hits.v); free(R->nt_cells.v); free(R->nt_n.v); free(R->nt_q.v);
  free(R->sv_idx.v); free(R->fit); free(R->near.v);
  free(R);
}
