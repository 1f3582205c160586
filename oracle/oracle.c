/*
 * CPU oracle for closest-hit / any-hit triangle BVH traversal.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h): used by the tests, the smoke check
 * and the benchmark's CPU baseline; never by the product path. Shares no code
 * with the CUDA library.
 *
 * Contents, each following the passage it cites:
 *  1. the pinned watertight ray/triangle test (Woop, Benthin & Wald, JCGT 2(1)
 *     2013), standing in for the paper's Moller-Trumbore test of App. G;
 *  2. brute-force closest-hit and any-hit: the plain definition;
 *  3. an independent binned-SAH BVH2 (Section 9.1: top-down SAH over binned
 *     centroids, here 32 bins) with the recursive closest_hit of Fig. 4 /
 *     App. G (test the box, cull on distmin, visit left then right, loop the
 *     leaf's triangles);
 *  4. the FP64 gradient of (t, u, v) with respect to the triangle and the ray,
 *     and its central-difference check.
 *
 * Build with -O2 -ffp-contract=off (no fast-math): the floating-point steps of
 * the intersector are part of its definition.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define MISS_ID 0xFFFFFFFFu

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int pick_threads(int threads) {
  return threads > 0 ? threads : oracle_max_threads();
}

/* ------------------------------------------------------------------ 1 */
/* Per-ray part of the watertight test: the axis kz of largest |d| (ties to the
 * lowest axis), kx, ky the next two cyclically (swapped when d[kz] < 0 to keep
 * the winding), and the shear constants Sx = d[kx]/d[kz], Sy = d[ky]/d[kz],
 * Sz = 1/d[kz]. */
typedef struct {
  int kx, ky, kz;
  float Sx, Sy, Sz;
} shear_t;

static void make_shear(const float *d, shear_t *s) {
  float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
  int kz = 0;
  float m = ax;
  if (ay > m) { kz = 1; m = ay; }
  if (az > m) { kz = 2; }
  int kx = (kz + 1) % 3;
  int ky = (kx + 1) % 3;
  if (d[kz] < 0.0f) { int tmp = kx; kx = ky; ky = tmp; }
  s->kx = kx; s->ky = ky; s->kz = kz;
  s->Sx = d[kx] / d[kz];
  s->Sy = d[ky] / d[kz];
  s->Sz = 1.0f / d[kz];
}

static int tri_finite(const float *p) {
  for (int k = 0; k < 9; ++k)
    if (!isfinite(p[k])) return 0;
  return 1;
}

/* The pinned test. A triangle with a non-finite vertex is never hit. The steps
 * and their rounding are fixed:
 *   A = p0 - o, B = p1 - o, C = p2 - o (componentwise);
 *   Ax = fma(-Sx, A[kz], A[kx]), Ay = fma(-Sy, A[kz], A[ky]), same for B, C;
 *   U = Cx*By - Cy*Bx, V = Ax*Cy - Ay*Cx, W = Bx*Ay - By*Ax (every product
 *   rounded to float, then the difference rounded);
 *   if any of U, V, W is zero, all three are recomputed from the exact double
 *   products and rounded back to float;
 *   miss if the signs of U, V, W differ (double-sided test);
 *   det = (U + V) + W, miss if zero;
 *   T = fma(W, Sz*C[kz], fma(V, Sz*B[kz], U*(Sz*A[kz])));
 *   t = T/det, u = V/det (weight of p1), v = W/det (weight of p2);
 *   accept iff max(tmin, 0) <= t <= tmax. The interval is closed at both
 *   ends, like the ray interval [tmin, tmax] of scion_ray. Its lower end is
 *   never below 0, so no hit behind the origin is reported, as in App. G,
 *   whose box test clamps the entry distance with max(0, .). App. G's
 *   triangle test is strict (t > 0): this reading differs from it only at
 *   t = 0 exactly, which it accepts when tmin <= 0. A NaN tmin counts as 0. */
static int tri_test(const float *o, const shear_t *s, float tmin, float tmax,
                    const float *p, float *t_out, float *u_out, float *v_out) {
  if (!tri_finite(p)) return 0;
  const int kx = s->kx, ky = s->ky, kz = s->kz;
  float A[3], B[3], C[3];
  for (int k = 0; k < 3; ++k) {
    A[k] = p[k] - o[k];
    B[k] = p[3 + k] - o[k];
    C[k] = p[6 + k] - o[k];
  }
  const float Ax = fmaf(-s->Sx, A[kz], A[kx]);
  const float Ay = fmaf(-s->Sy, A[kz], A[ky]);
  const float Bx = fmaf(-s->Sx, B[kz], B[kx]);
  const float By = fmaf(-s->Sy, B[kz], B[ky]);
  const float Cx = fmaf(-s->Sx, C[kz], C[kx]);
  const float Cy = fmaf(-s->Sy, C[kz], C[ky]);
  /* both products rounded, then subtracted: e(X, Y) = -e(Y, X) holds exactly,
   * so an edge shared by two triangles gets the same value with opposite sign
   * in both (watertightness); an FMA here would break that symmetry */
  const float CxBy = Cx * By, CyBx = Cy * Bx;
  const float AxCy = Ax * Cy, AyCx = Ay * Cx;
  const float BxAy = Bx * Ay, ByAx = By * Ax;
  float U = CxBy - CyBx;
  float V = AxCy - AyCx;
  float W = BxAy - ByAx;
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    double cxby = (double)Cx * (double)By, cybx = (double)Cy * (double)Bx;
    double axcy = (double)Ax * (double)Cy, aycx = (double)Ay * (double)Cx;
    double bxay = (double)Bx * (double)Ay, byax = (double)By * (double)Ax;
    U = (float)(cxby - cybx);
    V = (float)(axcy - aycx);
    W = (float)(bxay - byax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;
  const float det = (U + V) + W;
  if (det == 0.0f) return 0;
  const float Az = s->Sz * A[kz];
  const float Bz = s->Sz * B[kz];
  const float Cz = s->Sz * C[kz];
  const float UAz = U * Az;
  const float T = fmaf(W, Cz, fmaf(V, Bz, UAz));
  const float t = T / det;
  const float tlo = tmin > 0.0f ? tmin : 0.0f;
  if (!(t >= tlo && t <= tmax)) return 0;
  *t_out = t;
  *u_out = V / det;
  *v_out = W / det;
  return 1;
}

int oracle_intersect(const float *ray, const float *tri, float *t, float *u, float *v) {
  shear_t s;
  make_shear(ray + 4, &s);
  return tri_test(ray, &s, ray[3], ray[7], tri, t, u, v);
}

/* ------------------------------------------------------------------ 2 */
static void miss_hit(oracle_hit *h) {
  h->t = INFINITY;
  h->u = 0.0f;
  h->v = 0.0f;
  h->prim = MISS_ID;
}

/* Closest hit = lexicographic minimum of (t, id). */
static int better(float t, uint32_t id, float bt, uint32_t bid) {
  return t < bt || (t == bt && id < bid);
}

void oracle_closest_brute(const float *tris, uint64_t n_tris, const float *rays,
                          uint64_t n, oracle_hit *hits, int threads) {
  long long nn = (long long)n;
#pragma omp parallel for schedule(dynamic, 64) num_threads(pick_threads(threads))
  for (long long r = 0; r < nn; ++r) {
    const float *ray = rays + 8 * r;
    shear_t s;
    make_shear(ray + 4, &s);
    oracle_hit best;
    miss_hit(&best);
    for (uint64_t i = 0; i < n_tris; ++i) {
      float t, u, v;
      if (tri_test(ray, &s, ray[3], ray[7], tris + 9 * i, &t, &u, &v) &&
          better(t, (uint32_t)i, best.t, best.prim)) {
        best.t = t; best.u = u; best.v = v; best.prim = (uint32_t)i;
      }
    }
    hits[r] = best;
  }
}

void oracle_any_brute(const float *tris, uint64_t n_tris, const float *rays,
                      uint64_t n, uint32_t *occluded, int threads) {
  long long nn = (long long)n;
#pragma omp parallel for schedule(dynamic, 64) num_threads(pick_threads(threads))
  for (long long r = 0; r < nn; ++r) {
    const float *ray = rays + 8 * r;
    shear_t s;
    make_shear(ray + 4, &s);
    uint32_t occ = 0;
    for (uint64_t i = 0; i < n_tris && !occ; ++i) {
      float t, u, v;
      if (tri_test(ray, &s, ray[3], ray[7], tris + 9 * i, &t, &u, &v)) occ = 1;
    }
    occluded[r] = occ;
  }
}

/* ------------------------------------------------------------------ 3 */
/* Logical BVH2 (the paper's BVH ADT: Interior(left, right) | Leaf(prims),
 * each with bounds). Boxes are kept in double and padded outward by
 * BOX_PAD * (largest extent + largest |coordinate|), and the slab interval is
 * widened by T_MARGIN relative: far larger than any rounding in the float
 * intersector, so the traversal never culls a box holding an accepted hit. */
#define BOX_PAD 2.44140625e-4  /* 2^-12 */
#define T_MARGIN 2.44140625e-4

typedef struct {
  double lo[3], hi[3];
  uint32_t left, right;  /* children (interior) */
  uint32_t first, count; /* prim range (leaf iff count > 0) */
} onode;

struct oracle_bvh_s {
  onode *nodes;
  uint64_t n_nodes, cap;
  uint32_t *prim;   /* triangle ids in leaf order */
  float *tris;      /* private copy, [n_tris][9] */
  uint64_t n_tris;
  uint64_t n_used;  /* triangles in the tree (finite ones) */
  uint32_t depth;
};

typedef struct {
  double lo[3], hi[3];
} dbox;

static void box_empty(dbox *b) {
  for (int a = 0; a < 3; ++a) { b->lo[a] = INFINITY; b->hi[a] = -INFINITY; }
}
static void box_grow(dbox *b, const dbox *c) {
  for (int a = 0; a < 3; ++a) {
    if (c->lo[a] < b->lo[a]) b->lo[a] = c->lo[a];
    if (c->hi[a] > b->hi[a]) b->hi[a] = c->hi[a];
  }
}
static void box_grow_pt(dbox *b, const double *p) {
  for (int a = 0; a < 3; ++a) {
    if (p[a] < b->lo[a]) b->lo[a] = p[a];
    if (p[a] > b->hi[a]) b->hi[a] = p[a];
  }
}
static double box_area(const dbox *b) {
  double e[3];
  for (int a = 0; a < 3; ++a) e[a] = b->hi[a] > b->lo[a] ? b->hi[a] - b->lo[a] : 0.0;
  return 2.0 * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0]);
}

typedef struct {
  oracle_bvh *bvh;
  dbox *tbox;      /* per-triangle box */
  double *cent;    /* per-triangle centroid [3] */
  int bins, leaf_max;
} build_ctx;

static uint32_t new_node(oracle_bvh *b) {
  if (b->n_nodes == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 1024;
    b->nodes = (onode *)realloc(b->nodes, b->cap * sizeof(onode));
  }
  return (uint32_t)b->n_nodes++;
}

static void set_node_box(onode *nd, const dbox *b) {
  double ext = 0.0, mag = 0.0;
  for (int a = 0; a < 3; ++a) {
    double e = b->hi[a] - b->lo[a];
    if (e > ext) ext = e;
    if (fabs(b->lo[a]) > mag) mag = fabs(b->lo[a]);
    if (fabs(b->hi[a]) > mag) mag = fabs(b->hi[a]);
  }
  double pad = BOX_PAD * (ext + mag);
  for (int a = 0; a < 3; ++a) {
    nd->lo[a] = b->lo[a] - pad;
    nd->hi[a] = b->hi[a] + pad;
  }
}

static uint32_t build_rec(build_ctx *c, uint32_t first, uint32_t count, uint32_t depth) {
  oracle_bvh *b = c->bvh;
  if (depth > b->depth) b->depth = depth;
  uint32_t id = new_node(b);
  dbox nb, cb;
  box_empty(&nb);
  box_empty(&cb);
  for (uint32_t i = first; i < first + count; ++i) {
    uint32_t p = b->prim[i];
    box_grow(&nb, &c->tbox[p]);
    box_grow_pt(&cb, &c->cent[3 * p]);
  }
  set_node_box(&b->nodes[id], &nb);

  /* Binned SAH over the centroid bounds on every axis. */
  double best_cost = INFINITY;
  int best_axis = -1, best_split = -1;
  for (int a = 0; a < 3 && count > 1; ++a) {
    double ext = cb.hi[a] - cb.lo[a];
    if (!(ext > 0.0)) continue;
    int nb_ = c->bins;
    uint32_t cnt[64];
    dbox bb[64];
    for (int k = 0; k < nb_; ++k) { cnt[k] = 0; box_empty(&bb[k]); }
    double scale = nb_ / ext;
    for (uint32_t i = first; i < first + count; ++i) {
      uint32_t p = b->prim[i];
      int k = (int)((c->cent[3 * p + a] - cb.lo[a]) * scale);
      if (k >= nb_) k = nb_ - 1;
      if (k < 0) k = 0;
      cnt[k]++;
      box_grow(&bb[k], &c->tbox[p]);
    }
    double right_area[64];
    uint32_t right_cnt[64];
    dbox acc;
    box_empty(&acc);
    uint32_t n_acc = 0;
    for (int k = nb_ - 1; k > 0; --k) {
      box_grow(&acc, &bb[k]);
      n_acc += cnt[k];
      right_area[k] = box_area(&acc);
      right_cnt[k] = n_acc;
    }
    box_empty(&acc);
    n_acc = 0;
    for (int k = 0; k < nb_ - 1; ++k) {
      box_grow(&acc, &bb[k]);
      n_acc += cnt[k];
      if (n_acc == 0 || right_cnt[k + 1] == 0) continue;
      double cost = box_area(&acc) * n_acc + right_area[k + 1] * right_cnt[k + 1];
      if (cost < best_cost) { best_cost = cost; best_axis = a; best_split = k; }
    }
  }
  double leaf_cost = box_area(&nb) * count;
  double split_cost = box_area(&nb) + best_cost;  /* one traversal step + children */
  if (count == 1 || (count <= (uint32_t)c->leaf_max && (best_axis < 0 || leaf_cost <= split_cost))) {
    b->nodes[id].first = first;
    b->nodes[id].count = count;
    b->nodes[id].left = b->nodes[id].right = 0;
    return id;
  }
  uint32_t mid;
  if (best_axis < 0) {
    mid = first + count / 2;  /* all centroids coincide: split the range */
  } else {
    int a = best_axis;
    double scale = c->bins / (cb.hi[a] - cb.lo[a]);
    uint32_t i = first, j = first + count;
    while (i < j) {
      uint32_t p = b->prim[i];
      int k = (int)((c->cent[3 * p + a] - cb.lo[a]) * scale);
      if (k >= c->bins) k = c->bins - 1;
      if (k < 0) k = 0;
      if (k <= best_split) {
        ++i;
      } else {
        --j;
        uint32_t tmp = b->prim[i]; b->prim[i] = b->prim[j]; b->prim[j] = tmp;
      }
    }
    mid = i;
    if (mid == first || mid == first + count) mid = first + count / 2;
  }
  uint32_t l = build_rec(c, first, mid - first, depth + 1);
  uint32_t r = build_rec(c, mid, first + count - mid, depth + 1);
  b->nodes[id].left = l;
  b->nodes[id].right = r;
  b->nodes[id].first = 0;
  b->nodes[id].count = 0;
  return id;
}

oracle_bvh *oracle_bvh_build(const float *tris, uint64_t n_tris, int bins, int leaf_max) {
  if (bins < 2) bins = 2;
  if (bins > 64) bins = 64;
  if (leaf_max < 1) leaf_max = 1;
  oracle_bvh *b = (oracle_bvh *)calloc(1, sizeof(oracle_bvh));
  b->n_tris = n_tris;
  b->tris = (float *)malloc((n_tris ? n_tris : 1) * 9 * sizeof(float));
  memcpy(b->tris, tris, n_tris * 9 * sizeof(float));
  b->prim = (uint32_t *)malloc((n_tris ? n_tris : 1) * sizeof(uint32_t));
  build_ctx c;
  c.bvh = b;
  c.bins = bins;
  c.leaf_max = leaf_max;
  c.tbox = (dbox *)malloc((n_tris ? n_tris : 1) * sizeof(dbox));
  c.cent = (double *)malloc((n_tris ? n_tris : 1) * 3 * sizeof(double));
  uint64_t used = 0;
  for (uint64_t i = 0; i < n_tris; ++i) {
    const float *p = tris + 9 * i;
    if (!tri_finite(p)) continue;  /* never hit: left out of the tree */
    box_empty(&c.tbox[i]);
    for (int k = 0; k < 3; ++k) {
      double q[3] = {p[3 * k], p[3 * k + 1], p[3 * k + 2]};
      box_grow_pt(&c.tbox[i], q);
    }
    for (int a = 0; a < 3; ++a)
      c.cent[3 * i + a] = (p[a] + (double)p[3 + a] + p[6 + a]) / 3.0;
    b->prim[used++] = (uint32_t)i;
  }
  b->n_used = used;
  if (used > 0) build_rec(&c, 0, (uint32_t)used, 1);
  free(c.tbox);
  free(c.cent);
  return b;
}

void oracle_bvh_free(oracle_bvh *b) {
  if (!b) return;
  free(b->nodes);
  free(b->prim);
  free(b->tris);
  free(b);
}

void oracle_bvh_stats(const oracle_bvh *b, uint64_t *n_nodes, uint32_t *depth,
                      uint64_t *n_leaf_tris) {
  *n_nodes = b->n_nodes;
  *depth = b->depth;
  uint64_t s = 0;
  for (uint64_t i = 0; i < b->n_nodes; ++i) s += b->nodes[i].count;
  *n_leaf_tris = s;
}

/* Slab test in double against the padded box; returns 1 iff the widened
 * interval [max(tnear, tmin), min(tfar, tlim)] is non-empty. An axis with
 * d = 0 constrains only the origin coordinate. */
static int box_overlap(const onode *nd, const double *o, const double *rd,
                       const float *d, double tmin, double tlim) {
  double tn = -INFINITY, tf = INFINITY;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0f) {
      if (o[a] < nd->lo[a] || o[a] > nd->hi[a]) return 0;
      continue;
    }
    double t0 = (nd->lo[a] - o[a]) * rd[a];
    double t1 = (nd->hi[a] - o[a]) * rd[a];
    double n = t0 < t1 ? t0 : t1;
    double f = t0 < t1 ? t1 : t0;
    if (n > tn) tn = n;
    if (f < tf) tf = f;
  }
  tn -= T_MARGIN * fabs(tn);
  tf += T_MARGIN * fabs(tf);
  double lo = tn > tmin ? tn : tmin;
  double hi = tf < tlim ? tf : tlim;
  return lo <= hi;
}

typedef struct {
  const oracle_bvh *b;
  const float *ray;
  shear_t s;
  double o[3], rd[3];
  oracle_hit best;
  int any;       /* any-hit query */
  int found;
} trav_t;

static void visit(trav_t *q, uint32_t id) {
  const onode *nd = &q->b->nodes[id];
  double tlim = q->ray[7];
  if (!q->any && q->best.t < tlim) tlim = q->best.t;
  const double tlo = q->ray[3] > 0.0f ? q->ray[3] : 0.0;  /* as in tri_test */
  if (!box_overlap(nd, q->o, q->rd, q->ray + 4, tlo, tlim)) return;
  if (nd->count > 0) {
    for (uint32_t i = nd->first; i < nd->first + nd->count; ++i) {
      uint32_t p = q->b->prim[i];
      float t, u, v;
      if (!tri_test(q->ray, &q->s, q->ray[3], q->ray[7], q->b->tris + 9 * (uint64_t)p, &t, &u, &v))
        continue;
      if (q->any) { q->found = 1; return; }
      if (better(t, p, q->best.t, q->best.prim)) {
        q->best.t = t; q->best.u = u; q->best.v = v; q->best.prim = p;
      }
    }
    return;
  }
  visit(q, nd->left);
  if (q->any && q->found) return;
  visit(q, nd->right);
}

static void trace_one(const oracle_bvh *b, const float *ray, int any, trav_t *q) {
  q->b = b;
  q->ray = ray;
  q->any = any;
  q->found = 0;
  miss_hit(&q->best);
  make_shear(ray + 4, &q->s);
  for (int a = 0; a < 3; ++a) {
    q->o[a] = ray[a];
    q->rd[a] = 1.0 / (double)ray[4 + a];
  }
  if (b->n_nodes > 0) visit(q, 0);
}

void oracle_bvh_closest(const oracle_bvh *b, const float *rays, uint64_t n,
                        oracle_hit *hits, int threads) {
  long long nn = (long long)n;
#pragma omp parallel for schedule(dynamic, 64) num_threads(pick_threads(threads))
  for (long long r = 0; r < nn; ++r) {
    trav_t q;
    trace_one(b, rays + 8 * r, 0, &q);
    hits[r] = q.best;
  }
}

void oracle_bvh_any(const oracle_bvh *b, const float *rays, uint64_t n,
                    uint32_t *occluded, int threads) {
  long long nn = (long long)n;
#pragma omp parallel for schedule(dynamic, 64) num_threads(pick_threads(threads))
  for (long long r = 0; r < nn; ++r) {
    trav_t q;
    trace_one(b, rays + 8 * r, 1, &q);
    occluded[r] = (uint32_t)q.found;
  }
}

/* ------------------------------------------------------------------ 4 */
static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* The hit point satisfies o + t d = (1-u-v) p0 + u p1 + v p2, i.e. the linear
 * system [d | -e1 | -e2] (t, u, v) = p0 - o with e1 = p1 - p0, e2 = p2 - p0.
 * Solved by Cramer's rule. */
int oracle_plane_tuv(const double *o, const double *d, const double *p0,
                     const double *p1, const double *p2, double *tuv) {
  double c1[3], c2[3], r[3], x[3];
  for (int k = 0; k < 3; ++k) {
    c1[k] = -(p1[k] - p0[k]);
    c2[k] = -(p2[k] - p0[k]);
    r[k] = p0[k] - o[k];
  }
  cross3(c1, c2, x);
  double det = dot3(d, x);
  if (det == 0.0) return 0;
  double y[3], z[3];
  tuv[0] = dot3(r, x) / det;
  cross3(r, c2, y);
  tuv[1] = dot3(d, y) / det;
  cross3(c1, r, z);
  tuv[2] = dot3(d, z) / det;
  return 1;
}

static uint64_t vert_id(const uint32_t *tri_verts, uint64_t tri, int k) {
  return tri_verts ? (uint64_t)tri_verts[3 * tri + k] : 3 * tri + (uint64_t)k;
}

/* With J = [d | -e1 | -e2] and g = (dL/dt, dL/du, dL/dv), lambda solves
 * J^T lambda = g; then dL/do = -lambda, dL/dd = -t lambda, dL/dp0 =
 * (1-u-v) lambda, dL/dp1 = u lambda, dL/dp2 = v lambda (implicit function
 * theorem on o + t d - (1-u-v) p0 - u p1 - v p2 = 0). */
void oracle_grad(const float *tris, const uint32_t *tri_verts, uint64_t n_verts,
                 const float *rays, const oracle_hit *hits, const float *grad_tuv,
                 uint64_t n, double *grad_verts, double *grad_rays) {
  for (uint64_t r = 0; r < n; ++r) {
    double *gr = grad_rays ? grad_rays + 6 * r : NULL;
    if (gr) for (int k = 0; k < 6; ++k) gr[k] = 0.0;
    if (hits[r].prim == MISS_ID) continue;
    const uint64_t tri = hits[r].prim;
    const float *p = tris + 9 * tri;
    double d[3], c0[3], c1[3], c2[3];
    for (int k = 0; k < 3; ++k) {
      d[k] = rays[8 * r + 4 + k];
      c0[k] = d[k];
      c1[k] = -((double)p[3 + k] - p[k]);
      c2[k] = -((double)p[6 + k] - p[k]);
    }
    double x12[3], x20[3], x01[3];
    cross3(c1, c2, x12);
    cross3(c2, c0, x20);
    cross3(c0, c1, x01);
    double det = dot3(c0, x12);
    if (det == 0.0) continue;
    const double gt = grad_tuv[3 * r], gu = grad_tuv[3 * r + 1], gv = grad_tuv[3 * r + 2];
    double lam[3];
    for (int k = 0; k < 3; ++k) lam[k] = (gt * x12[k] + gu * x20[k] + gv * x01[k]) / det;
    const double t = hits[r].t, u = hits[r].u, v = hits[r].v;
    const double w[3] = {1.0 - u - v, u, v};
    for (int j = 0; j < 3; ++j) {
      uint64_t vid = vert_id(tri_verts, tri, j);
      if (vid >= n_verts) continue;
      for (int k = 0; k < 3; ++k) grad_verts[3 * vid + k] += w[j] * lam[k];
    }
    if (gr) {
      for (int k = 0; k < 3; ++k) {
        gr[k] = -lam[k];
        gr[3 + k] = -t * lam[k];
      }
    }
  }
}

static double loss_of(const double *o, const double *d, const double *p0,
                      const double *p1, const double *p2, const double *g) {
  double tuv[3];
  if (!oracle_plane_tuv(o, d, p0, p1, p2, tuv)) return 0.0;
  return g[0] * tuv[0] + g[1] * tuv[1] + g[2] * tuv[2];
}

void oracle_grad_fd(const float *tris, const uint32_t *tri_verts, uint64_t n_verts,
                    const float *rays, const oracle_hit *hits, const float *grad_tuv,
                    uint64_t n, double h, double *grad_verts, double *grad_rays) {
  for (uint64_t r = 0; r < n; ++r) {
    double *gr = grad_rays ? grad_rays + 6 * r : NULL;
    if (gr) for (int k = 0; k < 6; ++k) gr[k] = 0.0;
    if (hits[r].prim == MISS_ID) continue;
    const uint64_t tri = hits[r].prim;
    double x[15];  /* o, d, p0, p1, p2 */
    for (int k = 0; k < 3; ++k) {
      x[k] = rays[8 * r + k];
      x[3 + k] = rays[8 * r + 4 + k];
    }
    for (int k = 0; k < 9; ++k) x[6 + k] = tris[9 * tri + k];
    const double g[3] = {grad_tuv[3 * r], grad_tuv[3 * r + 1], grad_tuv[3 * r + 2]};
    double dx[15];
    for (int c = 0; c < 15; ++c) {
      double save = x[c];
      x[c] = save + h;
      double lp = loss_of(x, x + 3, x + 6, x + 9, x + 12, g);
      x[c] = save - h;
      double lm = loss_of(x, x + 3, x + 6, x + 9, x + 12, g);
      x[c] = save;
      dx[c] = (lp - lm) / (2.0 * h);
    }
    for (int j = 0; j < 3; ++j) {
      uint64_t vid = vert_id(tri_verts, tri, j);
      if (vid >= n_verts) continue;
      for (int k = 0; k < 3; ++k) grad_verts[3 * vid + k] += dx[6 + 3 * j + k];
    }
    if (gr) for (int k = 0; k < 6; ++k) gr[k] = dx[k];
  }
}

/* ------------------------------------------------------------------ closest point query
 * The paper's second traversal algorithm (App. G "Closest Point Query"): for a
 * query point p, the closest point on the closest triangle. The oracle fixes:
 *  - result = lexicographic minimum of (d2_i, i) over all triangles i with a
 *    finite vertex set and d2_i <= r2max (closed), d2_i the pinned squared
 *    distance below; a miss is d2 = +inf, u = v = 0, prim = 0xFFFFFFFF; a
 *    query point with a non-finite coordinate has no closest point (miss);
 *  - the closest point on a triangle by the Voronoi-region method of
 *    Ericson, Real-Time Collision Detection (2005), Section 5.1.5 (the
 *    reference App. G cites), in float with every product, sum and division
 *    rounded in the order written here:
 *      dot(x, y) = (x0*y0 + x1*y1) + x2*y2
 *      ab = b - a, ac = c - a, ap = p - a; d1 = dot(ab, ap), d2 = dot(ac, ap)
 *      vertex a: d1 <= 0 && d2 <= 0                        (u, v) = (0, 0)
 *      bp = p - b; d3 = dot(ab, bp), d4 = dot(ac, bp)
 *      vertex b: d3 >= 0 && d4 <= d3                        (1, 0)
 *      vc = d1*d4 - d3*d2
 *      edge ab: vc <= 0 && d1 >= 0 && d3 <= 0               s = d1/(d1 - d3); (s, 0), q = a + s*ab
 *      cp = p - c; d5 = dot(ab, cp), d6 = dot(ac, cp)
 *      vertex c: d6 >= 0 && d5 <= d6                        (0, 1)
 *      vb = d5*d2 - d1*d6
 *      edge ac: vb <= 0 && d2 >= 0 && d6 <= 0               s = d2/(d2 - d6); (0, s), q = a + s*ac
 *      va = d3*d6 - d5*d4
 *      edge bc: va <= 0 && d4 - d3 >= 0 && d5 - d6 >= 0    s = (d4 - d3)/((d4 - d3) + (d5 - d6));
 *                                                           (1 - s, s), q = b + s*(c - b)
 *      face: r = 1/((va + vb) + vc), v = vb*r, w = vc*r; (v, w), q = (a + ab*v) + ac*w
 *    (u, v) are the barycentric weights of p1 and p2 of the closest point.
 *    In the face case, v and w are first clamped to >= 0 and, if v + w > 1,
 *    both divided by (v + w): exact arithmetic never needs this, but with
 *    rounding the region tests can disagree with each other and the clamp
 *    keeps q inside the triangle;
 *      d2 = dot(p - q, p - q).
 * The paper's listing also lowers the bound with a "distmax" of each box;
 * that is not an upper bound on the distance to the nearest triangle for
 * boxes that are not tight, so neither side uses it. */
static float dot3f(const float *x, const float *y) { return (x[0] * y[0] + x[1] * y[1]) + x[2] * y[2]; }

static float closest_on_tri(const float *p, const float *tri, float *u_out, float *v_out) {
  const float *a = tri, *b = tri + 3, *c = tri + 6;
  float ab[3], ac[3], ap[3], bp[3], cp[3], q[3];
  for (int k = 0; k < 3; ++k) {
    ab[k] = b[k] - a[k];
    ac[k] = c[k] - a[k];
    ap[k] = p[k] - a[k];
  }
  float u, v;
  const float d1 = dot3f(ab, ap), d2 = dot3f(ac, ap);
  if (d1 <= 0.0f && d2 <= 0.0f) {
    u = 0.0f; v = 0.0f;
    for (int k = 0; k < 3; ++k) q[k] = a[k];
    goto done;
  }
  for (int k = 0; k < 3; ++k) bp[k] = p[k] - b[k];
  const float d3 = dot3f(ab, bp), d4 = dot3f(ac, bp);
  if (d3 >= 0.0f && d4 <= d3) {
    u = 1.0f; v = 0.0f;
    for (int k = 0; k < 3; ++k) q[k] = b[k];
    goto done;
  }
  const float vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
    const float s = d1 / (d1 - d3);
    u = s; v = 0.0f;
    for (int k = 0; k < 3; ++k) q[k] = a[k] + s * ab[k];
    goto done;
  }
  for (int k = 0; k < 3; ++k) cp[k] = p[k] - c[k];
  const float d5 = dot3f(ab, cp), d6 = dot3f(ac, cp);
  if (d6 >= 0.0f && d5 <= d6) {
    u = 0.0f; v = 1.0f;
    for (int k = 0; k < 3; ++k) q[k] = c[k];
    goto done;
  }
  const float vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
    const float s = d2 / (d2 - d6);
    u = 0.0f; v = s;
    for (int k = 0; k < 3; ++k) q[k] = a[k] + s * ac[k];
    goto done;
  }
  const float va = d3 * d6 - d5 * d4;
  const float e43 = d4 - d3, e56 = d5 - d6;
  if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
    const float s = e43 / (e43 + e56);
    u = 1.0f - s; v = s;
    for (int k = 0; k < 3; ++k) q[k] = b[k] + s * (c[k] - b[k]);
    goto done;
  }
  {
    const float r = 1.0f / ((va + vb) + vc);
    float fv = vb * r, fw = vc * r;
    if (!(fv >= 0.0f)) fv = 0.0f;
    if (!(fw >= 0.0f)) fw = 0.0f;
    const float sum = fv + fw;
    if (sum > 1.0f) {
      fv = fv / sum;
      fw = fw / sum;
    }
    u = fv; v = fw;
    for (int k = 0; k < 3; ++k) q[k] = (a[k] + ab[k] * fv) + ac[k] * fw;
  }
done:;
  float x[3];
  for (int k = 0; k < 3; ++k) x[k] = p[k] - q[k];
  *u_out = u;
  *v_out = v;
  return dot3f(x, x);
}

int oracle_closest_point(const float *pt, const float *tri, float *d2, float *u, float *v) {
  if (!tri_finite(tri)) return 0;
  *d2 = closest_on_tri(pt, tri, u, v);
  return 1;
}

void oracle_cpq_brute(const float *tris, uint64_t n_tris, const float *pts, uint64_t n,
                      oracle_hit *out, int threads) {
  long long nn = (long long)n;
#pragma omp parallel for schedule(dynamic, 64) num_threads(pick_threads(threads))
  for (long long r = 0; r < nn; ++r) {
    const float *p = pts + 4 * r;
    oracle_hit best;
    miss_hit(&best);
    /* a point that is not finite has no closest point */
    const int live = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
    for (uint64_t i = 0; live && i < n_tris; ++i) {
      const float *tri = tris + 9 * i;
      if (!tri_finite(tri)) continue;
      float u, v;
      const float d2 = closest_on_tri(p, tri, &u, &v);
      if (d2 <= p[3] && better(d2, (uint32_t)i, best.t, best.prim)) {
        best.t = d2; best.u = u; best.v = v; best.prim = (uint32_t)i;
      }
    }
    out[r] = best;
  }
}
