/*
 * CPU oracle for closest-hit / any-hit ray traversal of a triangle BVH.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may include, link or
 * call this code: only the test suite, the smoke check and the benchmark's CPU
 * baseline use it. It shares no code with the CUDA library.
 *
 * What it computes (the paper's problem statement, Fig. 4 and App. G
 * "Closest Hit Ray Tracing"): for each ray, the closest accepted
 * ray/triangle intersection, plus an any-hit predicate.
 *
 * Definitions the oracle fixes:
 *  - closest hit = lexicographic minimum of (t_i, i) over all triangles i
 *    accepted by the pinned watertight test (ties go to the lowest id);
 *  - any hit     = that set is non-empty;
 *  - a miss is reported as t = +inf, u = v = 0, prim = 0xFFFFFFFF.
 *
 * Layout of shared arguments:
 *  - tris : float [n_tris][9], p0.xyz p1.xyz p2.xyz in triangle-id order;
 *  - rays : float [n][8], (ox, oy, oz, tmin, dx, dy, dz, tmax);
 *  - hits : oracle_hit [n].
 * All buffers are host memory owned by the caller.
 */
#ifndef SCION_ORACLE_H
#define SCION_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  float t, u, v;
  uint32_t prim;
} oracle_hit;

typedef struct oracle_bvh_s oracle_bvh;

/* Pinned watertight intersection of one ray with one triangle. Returns 1 and
 * writes (t, u, v) on an accepted hit, else 0. */
int oracle_intersect(const float *ray, const float *tri, float *t, float *u, float *v);

/* Brute force over all triangles (OpenMP over rays; threads <= 0 = default). */
void oracle_closest_brute(const float *tris, uint64_t n_tris, const float *rays,
                          uint64_t n, oracle_hit *hits, int threads);
void oracle_any_brute(const float *tris, uint64_t n_tris, const float *rays,
                      uint64_t n, uint32_t *occluded, int threads);

/* Independent binned-SAH BVH2 and recursive traversal. */
oracle_bvh *oracle_bvh_build(const float *tris, uint64_t n_tris, int bins, int leaf_max);
void oracle_bvh_closest(const oracle_bvh *bvh, const float *rays, uint64_t n,
                        oracle_hit *hits, int threads);
void oracle_bvh_any(const oracle_bvh *bvh, const float *rays, uint64_t n,
                    uint32_t *occluded, int threads);
/* Node count, depth (root = 1), number of triangles referenced by leaves. */
void oracle_bvh_stats(const oracle_bvh *bvh, uint64_t *n_nodes, uint32_t *depth,
                      uint64_t *n_leaf_tris);
void oracle_bvh_free(oracle_bvh *bvh);

/* FP64 gradient of L = sum_i g_t,i t_i + g_u,i u_i + g_v,i v_i with every
 * ray's hit triangle held fixed. grad_tuv: float [n][3]. tri_verts: uint32
 * [n_tris][3] vertex ids (NULL for a soup: vertex 3*i+k). grad_verts: double
 * [n_verts][3], accumulated (+=). grad_rays: double [n][6] (o, d), overwritten;
 * missed rays get zeros. */
void oracle_grad(const float *tris, const uint32_t *tri_verts, uint64_t n_verts,
                 const float *rays, const oracle_hit *hits, const float *grad_tuv,
                 uint64_t n, double *grad_verts, double *grad_rays);

/* The same gradient by central differences of the FP64 plane intersection
 * (no inside test, triangle fixed), step h. Same output convention. */
void oracle_grad_fd(const float *tris, const uint32_t *tri_verts, uint64_t n_verts,
                    const float *rays, const oracle_hit *hits, const float *grad_tuv,
                    uint64_t n, double h, double *grad_verts, double *grad_rays);

/* FP64 plane intersection (t, u, v) of a ray with a fixed triangle. Returns 0
 * if the ray is parallel to the plane. */
int oracle_plane_tuv(const double *o, const double *d, const double *p0,
                     const double *p1, const double *p2, double *tuv);

/* Closest point query (App. G): for each point (x, y, z, r2max) the
 * lexicographic minimum of (d2, id) over triangles with d2 <= r2max, d2 the
 * squared distance to the pinned closest point on the triangle (Ericson 2005,
 * Section 5.1.5; see oracle.c). out[i] = {d2, u, v, prim}: (u, v) weights of
 * p1 and p2 of the closest point; miss = {inf, 0, 0, 0xFFFFFFFF}. */
void oracle_cpq_brute(const float *tris, uint64_t n_tris, const float *pts, uint64_t n,
                      oracle_hit *out, int threads);
/* One point (3 floats) against one triangle; 0 if the triangle is not finite. */
int oracle_closest_point(const float *pt, const float *tri, float *d2, float *u, float *v);

int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
