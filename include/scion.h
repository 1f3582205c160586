/*
 * scion.h — C ABI of the GB300 (sm_103a) closest-hit / any-hit traversal
 * library for triangle BVHs whose physical data layout is chosen separately
 * from one traversal loop.
 *
 * The calls follow the paper's statement of the problem (Section 3, Fig. 4 and
 * App. G "Closest Hit Ray Tracing": a Ray, a logical BVH over triangles, and
 * the closest_hit query) and its decoupling of physical layout from traversal
 * (Section 4, the layout language; Section 5, two-phase build; Table 1, the
 * evaluated layouts).
 *
 * General conventions
 *  - Every call returns a scion_status; no call aborts, traps or throws.
 *  - Argument and descriptor errors are reported synchronously and nothing is
 *    launched.
 *  - Trace calls are asynchronous on the given stream. They never synchronise
 *    the host. Errors found on the device (stack overflow, step limit) are
 *    recorded in the BVH's device status word and the affected ray's hit gets
 *    prim = SCION_PRIM_ERROR; scion_get_status reads and clears that word.
 *  - Device pointers are CUDA device addresses on the current device. A BVH
 *    is used on the device it was built on: a call on it while another
 *    device is current, or with device memory of another GPU, returns
 *    SCION_ERR_INVALID_ARG before anything is issued.
 *  - scion_last_error() holds the message of the last failing call of the
 *    calling host thread.
 *  - Rays and hits are caller-owned. The BVH owns its own device buffers.
 *  - One BVH may be traced concurrently from up to 64 distinct streams: each
 *    stream gets its own work counter in the BVH (calls on one stream run in
 *    order). A 65th stream is refused with SCION_ERR_INVALID_ARG.
 */
#ifndef SCION_H
#define SCION_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *scion_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  SCION_OK = 0,
  SCION_ERR_INVALID_ARG = 1,
  SCION_ERR_UNSUPPORTED_LAYOUT = 2,
  SCION_ERR_OOM = 3,
  SCION_ERR_CUDA = 4,
  SCION_ERR_STACK_OVERFLOW = 5,
  SCION_ERR_ITER_LIMIT = 6,
  SCION_ERR_BAD_INPUT = 7
} scion_status;

#define SCION_PRIM_MISS 0xFFFFFFFFu
#define SCION_PRIM_ERROR 0xFFFFFFFEu

/* Layout descriptor: the physical representation of one logical BVH
 * (Section 4 layout primitives: node arity, group AoS/SoA (Section 4.2.2),
 * quantised derived bounds (Section 4.2.1, App. D.2), bit-stolen or indirect
 * references (split / indirect group ... from, Section 4.2.2-4.2.3), and the
 * build order attribute order=pre (Section 5.3.2)).
 *
 *  width      : 2, 4 or 8 children per node.
 *  box_layout : 0 AoS, 1 SoA. For width 2 with f32 boxes the node stores its
 *               own box (the PBRTv4 LinearBVH of Fig. 4b, 32 B per node);
 *               SoA then splits boxes and references into two arrays. For all
 *               other layouts child boxes are stored in the parent node,
 *               interleaved per child (AoS) or per coordinate (SoA).
 *  box_prec   : 0 f32, 1 f16 (world frame, rounded outward),
 *               2 u8 (relative to the parent's merged box, rounded outward,
 *               App. D.2 reading). f16/u8 need a children-in-parent node.
 *               3 q16 and 4 eq10: width-2 own-box nodes whose box is stored
 *               as integer codes on one grid over the root box ("sg-pbrt-q16"
 *               of Section 9.2.5 / App. D.3: 16-bit codes, 16 B per node;
 *               "sg-eq" of App. D.1: 10-bit codes, 12 B per node). Codes are
 *               chosen so that the decoded box encloses the node's box.
 *               These need leaf_max <= 15 and fewer than 2^26 nodes; q16
 *               takes AoS or SoA ("-soaos": code array + word array), eq10
 *               AoS only.
 *               5 u16: children-in-parent codes relative to the parent's
 *               merged box like u8, 16 bits each (bvh8-q16 of Table 1).
 *               6 shared slab (Section 8.3): width-2 node without a box: the
 *               split axis and two planes (the left child's upper and the
 *               right child's lower bound on that axis), 16 B; children
 *               inherit the other planes from the parent's box, which the
 *               traversal carries from the root. AoS only; not for closest
 *               point queries (SCION_ERR_UNSUPPORTED_LAYOUT there).
 *  child_ref  : 0 direct (an explicit reference per child; for the width-2
 *               own-box node: implicit left = I+1 and stored right offset,
 *               which requires order = DFS), 1 indirect (one base index,
 *               siblings stored contiguously).
 *  prim_ref   : 0 direct (triangles copied in leaf order, 48 B each),
 *               1 indirect (a 32-bit triangle id per leaf entry into the BVH's
 *               vertex/index tables).
 *  order      : 0 DFS pre-order, 1 BFS, 2 treelet (greedy, surface-area
 *               ordered clusters of at most treelet_bytes).
 *  leaf_max   : triangles per leaf, 1..16 (0 = 4).
 *  sah_bins   : SAH bins, 2..64 (0 = 16).
 *  treelet_bytes : treelet budget in bytes (0 = 1024).
 *  align      : 0 or 16. 16 pads each own-box node record (or SoA box
 *               record) to a multiple of 16 bytes ("-align16" of Table 1:
 *               eq10 12 -> 16 B, q16 SoA codes 12 -> 16 B, f32 SoA boxes
 *               24 -> 32 B); layouts already 16-byte multiples are unchanged.
 *               Other values: SCION_ERR_INVALID_ARG.
 * Unsupported combinations return SCION_ERR_UNSUPPORTED_LAYOUT. */
typedef struct {
  uint32_t width;
  uint32_t box_layout;
  uint32_t box_prec;
  uint32_t child_ref;
  uint32_t prim_ref;
  uint32_t order;
  uint32_t leaf_max;
  uint32_t sah_bins;
  uint32_t treelet_bytes;
  uint32_t align;
} scion_layout_desc;

/* A ray (the paper's Ray of Fig. 4 with an added tmin): accepted hits satisfy
 * tmin <= t <= tmax. 32 bytes, 16-byte aligned arrays. */
typedef struct {
  float ox, oy, oz, tmin;
  float dx, dy, dz, tmax;
} scion_ray;

/* A closest hit: t, barycentric weights u (of p1) and v (of p2), and the
 * caller's triangle index. A miss is t = +inf, u = v = 0,
 * prim = SCION_PRIM_MISS. 16 bytes. */
typedef struct {
  float t, u, v;
  uint32_t prim;
} scion_hit;

/* Traversal parameters; NULL or 0 fields = defaults.
 *  threads_per_block : CTA size (multiple of 32, <= 1024; default 256).
 *  ctas_per_sm       : persistent CTAs per SM (default: from occupancy).
 *  reg_stack         : entries of the traversal stack kept in registers
 *                      (0, 2 or 4; default 0): the newest entries stay in
 *                      registers and older ones move to the shared-memory
 *                      part (then local memory), which saves a shared-memory
 *                      store and load per entry that is popped while still
 *                      in registers. The paper's traversal uses a 64-entry
 *                      stack (Section 9.2). Results are identical. Other
 *                      values, or a non-zero value for closest point
 *                      queries: SCION_ERR_INVALID_ARG.
 *  smem_stack        : shared-memory stack entries per thread (default 16,
 *                      at most 64; traces of own-box bvh2 layouts other than
 *                      the shared slab and of 2/4-wide layouts round it down
 *                      to a power of two).
 *  ordered_children  : 0 or 1 = children sorted by entry distance
 *                      (closest hit), 2 = stored slot order, 3 = nearest
 *                      child first and the others in slot order.
 *  rays_per_fetch    : 0 (or 32) = each warp takes 32 consecutive rays and
 *                      traces them to completion; k in 1..31 = a warp
 *                      refills its idle lanes as soon as at least k of them
 *                      are idle (32-ray blocks are dealt to the CTAs
 *                      round-robin, rays handed out from a shared-memory
 *                      counter; k = 1 refills a lane at the next step).
 *                      Results are identical; which is faster depends on the
 *                      layout and the rays. Above 32: SCION_ERR_INVALID_ARG.
 *  max_steps         : per-ray node+leaf visit limit (0 = derived from size).
 *  raster_width      : 0, or the rays are a row-major image this many rays
 *                      wide (ray i is pixel (i mod w, i / w); the last row
 *                      may be partial): each warp then traces an 8 x 4 pixel
 *                      tile instead of 32 consecutive rays, which keeps camera
 *                      rays of one warp close together. Warp batches only
 *                      (rays_per_fetch 0 or 32), rays only (not closest point
 *                      queries), not in batched launches; otherwise
 *                      SCION_ERR_INVALID_ARG. Results are identical. */
typedef struct {
  uint32_t threads_per_block, ctas_per_sm, reg_stack, smem_stack, ordered_children,
      rays_per_fetch, max_steps, raster_width;
} scion_trace_params;

/* A closest point query (App. G "Closest Point Query"): a point and a squared
 * search radius; only triangles with d2 <= r2max count (+inf: unbounded).
 * 16 bytes, 16-byte aligned arrays. */
typedef struct {
  float x, y, z, r2max;
} scion_point;

/* A closest point: squared distance d2 to the closest point on triangle
 * `prim`, whose barycentric weights of p1 and p2 are u and v. A miss (no
 * triangle within the radius, or a point that is not finite) is d2 = +inf,
 * u = v = 0, prim = SCION_PRIM_MISS. 16 bytes. */
typedef struct {
  float d2, u, v;
  uint32_t prim;
} scion_closest_point;

typedef struct scion_bvh_s *scion_bvh;

/* Build a BVH (Section 5.1 two-phase construction: binned-SAH logical BVH2,
 * Section 9.1; collapse to the requested width; order; count pass, one
 * allocation per buffer, fill pass, App. F) and upload it.
 *  verts   : float [n_verts][3], host or device memory (read, not retained).
 *  indices : uint32 [n_tris][3] or NULL for a soup (triangle i = vertices
 *            3i..3i+2, n_verts must be 3*n_tris). Host or device memory.
 *  desc    : layout descriptor (host).
 *  stream  : stream for the uploads; the call returns after they complete.
 *  out     : receives the handle; *out is NULL on error.
 * Triangles with a non-finite vertex are never hit and are left out.
 * Errors: INVALID_ARG (null pointers, index out of range, n_tris >= 2^27),
 * UNSUPPORTED_LAYOUT, OOM, CUDA. */
scion_status scion_build(const float *verts, uint64_t n_verts, const uint32_t *indices,
                         uint64_t n_tris, const scion_layout_desc *desc, scion_stream stream,
                         scion_bvh *out);

/* Several layouts of one scene from a single logical build (Section 5.1: the
 * topology is fixed first, then packed into each physical layout). descs:
 * n_desc descriptors that must agree on leaf_max and sah_bins (else
 * INVALID_ARG); out: n_desc handles, all NULL on error. Other arguments and
 * errors as scion_build. */
scion_status scion_build_many(const float *verts, uint64_t n_verts, const uint32_t *indices,
                              uint64_t n_tris, const scion_layout_desc *descs, uint32_t n_desc,
                              scion_stream stream, scion_bvh *out);

/* The same as scion_build, but the logical BVH2 is constructed on the GPU
 * (Section 5.1 keeps construction apart from the layout build; Section 2:
 * topology is orthogonal to layout) as a linear BVH: 30-bit Morton codes of
 * the triangle centroids, a stable radix sort, the binary radix tree of
 * Karras (2012) and boxes bottom-up; a subtree of at most leaf_max triangles
 * becomes one leaf where the surface area heuristic prefers it to splitting
 * (sah_bins is not used). The tree is then packed
 * into `desc` by the same host packers as scion_build.
 *  d_verts   : float [n_verts][3], DEVICE memory (read, not retained).
 *  d_indices : uint32 [n_tris][3] in DEVICE memory, or NULL for a soup.
 *  stream    : stream for the build kernels and copies; the call returns
 *              after they complete.
 * Device scratch of about 60 bytes per triangle is allocated for the
 * duration of the call. Errors as scion_build; host pointers give
 * INVALID_ARG. */
scion_status scion_build_gpu(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices,
                             uint64_t n_tris, const scion_layout_desc *desc, scion_stream stream,
                             scion_bvh *out);

/* Refit to new vertex positions: same triangles, same indices, same tree.
 * Every node's box is recomputed bottom-up from the new vertices and
 * re-encoded in place in the BVH's layout (the same codecs as the build,
 * rounded outward, with the build pad), and the BVH's vertex table and
 * direct triangle copies are rewritten. Results of later traces are those of
 * the moved scene; tree quality degrades as the motion grows (rebuild then).
 * Triangles left out at build time (non-finite) stay out; a triangle whose
 * vertex becomes non-finite is never hit.
 *  d_verts : float [n_verts][3], DEVICE memory; n_verts must equal the
 *            BVH's vertex count.
 *  stream  : the refit kernels run on it, asynchronously, except for the
 *            world-grid layouts (q16, eq10) and the shared-slab layout,
 *            whose new grid or root box is read back (the call then
 *            synchronises the stream).
 * No trace of this BVH may run concurrently on another stream. The first
 * call allocates about 32 bytes of device scratch per node, kept until
 * scion_destroy. A box code that cannot enclose its box sets the device
 * status word to SCION_ERR_BAD_INPUT (scion_get_status).
 * Errors: INVALID_ARG (null, host memory, vertex count), OOM, CUDA. */
scion_status scion_refit(scion_bvh bvh, const float *d_verts, uint64_t n_verts, scion_stream stream);

/* Build timings of a BVH in milliseconds: logical_ms = construction of the
 * logical BVH2 (host wall time of the binned-SAH builder, or device time of
 * scion_build_gpu's kernels); pack_ms = host packing into the layout. Either
 * pointer may be NULL. */
scion_status scion_bvh_build_times(scion_bvh bvh, double *logical_ms, double *pack_ms);

/* Sizes of the device buffers (bytes) and tree shape. Any output pointer may
 * be NULL. node_bytes: node buffer(s); prim_bytes: leaf primitive buffer
 * (direct triangles, or ids plus the index table for indirect); depth: levels
 * of the stored tree; n_nodes: stored nodes. */
scion_status scion_bvh_info(scion_bvh bvh, uint64_t *node_bytes, uint64_t *prim_bytes,
                            uint32_t *depth, uint32_t *n_nodes);

/* Closest hit of each ray (Fig. 4 closest_hit; ties at equal t go to the
 * lowest triangle index). d_rays: scion_ray[n]; d_hits: scion_hit[n]; each in
 * device memory or in page-locked host memory (cudaHostAlloc,
 * cudaHostRegister), which the kernel then reads or writes in place over the
 * host link, with no staging copy; results in host memory are complete once
 * `stream` has reached the end of the call. Pageable host memory:
 * SCION_ERR_INVALID_ARG, before any launch. params: NULL for defaults. n = 0
 * is a no-op. */
scion_status scion_trace_closest(scion_bvh bvh, const scion_ray *d_rays, uint64_t n,
                                 scion_hit *d_hits, const scion_trace_params *params,
                                 scion_stream stream);

/* Any hit: d_occluded[i] = 1 iff ray i has an accepted hit in [tmin, tmax],
 * else 0 (uint32[n]). Buffers as for scion_trace_closest. */
scion_status scion_trace_any(scion_bvh bvh, const scion_ray *d_rays, uint64_t n,
                             uint32_t *d_occluded, const scion_trace_params *params,
                             scion_stream stream);

/* Backward pass of scion_trace_closest (no counterpart in the paper, which
 * has no gradient). Each hit ray's triangle is held fixed (the traversal's
 * discrete choice); dL/d(t,u,v) is carried through the hit-point identity
 * o + t d = (1-u-v) p0 + u p1 + v p2 to the triangle's three vertices and to
 * the ray.
 *  d_rays, d_hits : the forward call's rays and hits (device, n each).
 *  d_grad_tuv     : device float[n][3], dL/dt, dL/du, dL/dv per ray.
 *  d_grad_verts   : device float[n_verts][3] in the vertex order given to
 *                   scion_build; contributions are ADDED (FP32 atomics, so the
 *                   summation order, and the last bits, vary between runs).
 *  d_grad_rays    : device scion_ray-shaped float[n][8] receiving dL/d(o, d)
 *                   (tmin and tmax entries are 0), or NULL.
 * Missed rays (prim = SCION_PRIM_MISS) and errored rays contribute nothing.
 * The per-ray 3x3 solve is done in double precision. Every buffer must be
 * device memory (the gradients are scattered with device atomics), else
 * SCION_ERR_INVALID_ARG. */
scion_status scion_trace_backward(scion_bvh bvh, const scion_ray *d_rays, const scion_hit *d_hits,
                                  const float *d_grad_tuv, uint64_t n, float *d_grad_verts,
                                  scion_ray *d_grad_rays, scion_stream stream);

/* Closest point on the scene for each query point (App. G "Closest Point
 * Query", on any layout of the BVH): the lexicographic minimum of (d2, id)
 * over the triangles with d2 <= r2max, d2 the squared distance to the closest
 * point on the triangle by the Voronoi-region method (Ericson 2005, Section
 * 5.1.5) in float with a fixed rounding order (results are identical on
 * every layout). Node boxes are bounded from below with outward rounding, so
 * no box that could hold the winner is skipped; the paper's "distmax" bound
 * update is not used.
 *  d_points : scion_point[n] (16-byte aligned), device or page-locked host
 *             memory as for scion_trace_closest.
 *  d_out    : scion_closest_point[n] (16-byte aligned), likewise.
 *  params   : as scion_trace_closest (ordered_children: 0/1 children sorted
 *             by box distance, 2 slot order, 3 nearest first); rays_per_fetch
 *             must be 0 or 32.
 * Asynchronous on `stream`; errors and device status as scion_trace_closest. */
scion_status scion_query_closest_point(scion_bvh bvh, const scion_point *d_points, uint64_t n,
                                      scion_closest_point *d_out, const scion_trace_params *params,
                                      scion_stream stream);

/* Counting variant of the traces, for measurement: the same results
 * (query 0: closest hits into scion_hit[n]; query 1: any-hit flags into
 * uint32[n]; query 2: closest points, d_rays then holding scion_point[n] and
 * d_out scion_closest_point[n]) plus visit counters added into d_counters
 * (device uint64[4], else SCION_ERR_INVALID_ARG): [0] interior nodes fetched, [1] leaves visited,
 * [2] triangles tested, [3] rays (points) traced. Slower than the plain
 * calls; not for production use. */
scion_status scion_trace_stats(scion_bvh bvh, const scion_ray *d_rays, uint64_t n, uint32_t query,
                               void *d_out, const scion_trace_params *params, scion_stream stream,
                               uint64_t *d_counters);

/* Closest hit for callers that cannot allocate device memory when they
 * trace: an application that hands all device memory to its own arena up
 * front and forbids any later allocation, or a latency-bound thread that must
 * not enter the driver's allocator (cudaMalloc can synchronize the device and
 * take milliseconds). The paper has no counterpart; this is a property of
 * this library only.
 *
 * Same arguments and results as scion_trace_closest (the BVH, rays and hits
 * are the caller's, built and allocated beforehand). The traversal's work
 * counters live in a fixed 256-byte device array that the library reserves
 * on every GPU that loads it, for the life of the process; 16 bytes of it are
 * used. The call allocates nothing and frees nothing: it clears those 16
 * bytes with cudaMemsetAsync on `stream` and launches the kernel.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress), so make that first call before any stream
 *    capture begins.
 *  - Every call on a device shares the one array: calls that overlap on the
 *    GPU (different streams, or concurrent graphs) race and give wrong
 *    results. Order them on one stream.
 *  - Device errors still set the BVH's status word (scion_get_status).
 *  - n >= 2^62 is rejected with SCION_ERR_INVALID_ARG (the counter in the
 *    array must not wrap); scion_last_error() names the limit. */
scion_status scion_trace_closest_noalloc(scion_bvh bvh, const scion_ray *d_rays, uint64_t n,
                                         scion_hit *d_hits, const scion_trace_params *params,
                                         scion_stream stream);

/* ---- Many scenes in one launch (closest hit). No counterpart in the paper,
 * whose measurements (Section 9.2) show the best layout changes with the
 * workload; this lets each scene keep the layout chosen for it while all of
 * them run in one persistent launch.
 *
 * scion_batch_create records scene i = (bvhs[i], d_rays[i] (scion_ray[n[i]]),
 * d_hits[i] (scion_hit[n[i]]), both device or page-locked host memory as for
 * scion_trace_closest, per_scene[i] or
 * defaults) into a device table (it allocates and uploads; synchronous on
 * `stream`). threads_per_block and smem_stack are taken from per_scene[0];
 * each scene's ordered_children, rays_per_fetch (warp batches or warp
 * refill, applied within the 256-ray chunks a warp takes) and max_steps are
 * its own. raster_width and reg_stack are plain-launch parameters: non-zero
 * values give SCION_ERR_INVALID_ARG.
 * Scenes whose layout is one of the batched node families (width-2 own-box
 * AoS with f32 or q16 boxes, width-4 SoA with f32, f16 or u8 boxes, width-8
 * SoA f16, width-8 u8 AoS or SoA, each with direct child references;
 * triangles direct or indirect) run in one persistent kernel; any other scene
 * gets its own plain launch from scion_batch_launch.
 * The pointers are captured: the buffers must stay valid until the batch is
 * destroyed.
 *
 * scion_batch_launch issues the work on `stream`: no allocation, no host
 * synchronisation, so it may be captured into a CUDA graph and replayed.
 * Results are identical to scion_trace_closest on each scene. Launches of one
 * batch must not overlap on the GPU (they share its counters). */
typedef struct scion_batch_s *scion_batch;
scion_status scion_batch_create(const scion_bvh *bvhs, const scion_ray *const *d_rays, const uint64_t *n,
                                scion_hit *const *d_hits, uint32_t n_scenes,
                                const scion_trace_params *per_scene, scion_stream stream,
                                scion_batch *out);
scion_status scion_batch_launch(scion_batch batch, scion_stream stream);
/* Scenes in the single multi-scene launch / scenes traced by plain launches. */
scion_status scion_batch_info(scion_batch batch, uint32_t *batched_scenes, uint32_t *plain_scenes);
void scion_batch_destroy(scion_batch batch);

/* One-shot form: create, launch, wait for the stream, destroy. */
scion_status scion_trace_batched(const scion_bvh *bvhs, const scion_ray *const *d_rays, const uint64_t *n,
                                 scion_hit *const *d_hits, uint32_t n_scenes,
                                 const scion_trace_params *per_scene, scion_stream stream);

/* Device status of the BVH since the last call: synchronises the stream,
 * returns SCION_OK or the first device-side error code, and clears it. */
scion_status scion_get_status(scion_bvh bvh, scion_stream stream, scion_status *device_status);

void scion_destroy(scion_bvh bvh);

const char *scion_status_string(scion_status s);

#ifdef __cplusplus
}
#endif
#endif
