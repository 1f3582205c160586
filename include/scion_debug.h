/*
 * scion_debug.h — introspection entry points of the scion library, used by
 * the test suite to check the packer and the codecs without a GPU.
 *
 * The paper's round-trip property (App. B, "Round-Trip Soundness": decoding
 * an encoded tree gives back the logical tree) is checked through these
 * calls: a host-only build packs a scene exactly as scion_build does, and the
 * decode call reads every packed node back into its logical view (child
 * kind, child node or leaf range, conservative box).
 *
 * All pointers here are host memory owned by the caller, and none of these
 * calls touches a GPU, except scion_debug_read_bandwidth (a measurement
 * probe, device memory), scion_debug_build_gpu_host_pack and
 * scion_debug_bvh_bytes (the GPU packer's reference and its check).
 */
#ifndef SCION_DEBUG_H
#define SCION_DEBUG_H

#include <stdint.h>

#include "scion.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scion_host_bvh_s *scion_host_bvh;

typedef struct {
  uint32_t n_nodes;        /* stored nodes */
  uint32_t node_stride;    /* bytes per node in the (first) node array */
  uint32_t n_leaf_entries; /* triangles referenced by leaves */
  uint32_t root_ref;       /* encoded root reference (wide) or 0 (own-box) */
  uint32_t depth;          /* levels of the stored tree */
  uint32_t stack_need;     /* worst-case traversal stack entries */
  uint32_t own_box;        /* 1 = width-2 own-box node */
  uint32_t node2_bytes;    /* second node array (own-box SoA words/refs), bytes */
  uint64_t node_bytes;     /* node buffer(s) */
  uint64_t prim_bytes;     /* leaf primitive buffer (+ index table if indirect) */
  uint64_t vert_bytes;     /* float4 vertex table */
  double build_ms;         /* host build + pack time */
} scion_debug_info;

/* Build and pack on the host only (same code path as scion_build, no upload).
 * verts/indices: host arrays as in scion_build. Errors as scion_build. */
scion_status scion_debug_build_host(const float *verts, uint64_t n_verts, const uint32_t *indices,
                                    uint64_t n_tris, const scion_layout_desc *desc,
                                    scion_host_bvh *out);

scion_status scion_debug_host_stats(scion_host_bvh hb, scion_debug_info *info);

/* Decode every packed node. Arrays sized for n_nodes * 8 child slots:
 *  kind[i*8+k]   : 0 empty, 1 interior, 2 leaf (own-box nodes: slots 0-1 are
 *                  the two children (kind 1), or slot 0 is the node's own
 *                  leaf range (kind 2));
 *  a[i*8+k]      : child node index (interior) or first leaf entry (leaf);
 *  c[i*8+k]      : leaf entry count (leaf) else 0;
 *  boxes[(i*8+k)*6..]: decoded child box lo.xyz, hi.xyz (wide nodes);
 *  own_boxes[i*6..]  : the node's own box (own-box nodes);
 *  leaf_ids[j]   : triangle id of leaf entry j (n_leaf_entries values). */
scion_status scion_debug_host_decode(scion_host_bvh hb, uint32_t *kind, uint32_t *a, uint32_t *c,
                                     float *boxes, float *own_boxes, uint32_t *leaf_ids);

/* Raw packed bytes: the node array (n_nodes * node_stride bytes), the second
 * node array (node2_bytes; own-box SoA only) and the nine floats of the
 * world grid of the quantised own-box codecs (q16: wlo.xyz, step.xyz, 0, 0,
 * 0; eq10: wlo.xyz, whi.xyz, bin.xyz; zeros for other layouts), so a test can
 * decode the codes on its own. SCION_ERR_INVALID_ARG if a capacity (bytes)
 * is too small. */
scion_status scion_debug_host_raw(scion_host_bvh hb, void *nodes, uint64_t nodes_cap, void *nodes2,
                                  uint64_t nodes2_cap, float *frame);

void scion_debug_host_destroy(scion_host_bvh hb);

/* Directed rounding of a float to IEEE binary16 (dir < 0: toward -inf,
 * dir > 0: toward +inf), returned as the 16 bits; and the exact decode. */
uint32_t scion_debug_f16_round(float x, int dir);
float scion_debug_f16_decode(uint32_t h);

/* Warp-batch slots of a launch over n rays with the traversal parameter
 * raster_width = w (0: n; else 32 per 8 x 4 pixel tile, up to the last tile
 * that holds a ray): the loop bound the trace kernels get. Host only. */
uint64_t scion_debug_raster_slots(uint64_t n, uint32_t raster_width);

/* Measurement probe for the roofline of traversals whose BVH fits in L2 (the
 * bandwidth bound of Section 9.2's finding that compact layouts win by moving
 * fewer bytes): one launch that reads the device buffer d_buf (bytes, a
 * multiple of 16, 16-byte aligned) `reps` times with 16-byte loads that
 * bypass L1 (ld.global.cg), from every SM, asynchronously on `stream`. A
 * buffer well below the L2 size stays in L2, so bytes * reps / (launch time)
 * is the L2 read bandwidth; the caller times the launch (CUDA events on
 * `stream`). d_sink: device uint32 that the kernel may write (it keeps the
 * loads from being optimised away; its value means nothing). Both buffers
 * must be device memory of the current device, else SCION_ERR_INVALID_ARG. */
scion_status scion_debug_read_bandwidth(const void *d_buf, uint64_t bytes, uint32_t reps, uint32_t *d_sink,
                                        scion_stream stream);

/* The GPU construction of scion_build_gpu with the packing done by the host
 * packers instead of the GPU packer (arguments, errors and result as
 * scion_build_gpu): the reference against which the GPU packer's bytes are
 * compared. */
scion_status scion_debug_build_gpu_host_pack(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices,
                                             uint64_t n_tris, const scion_layout_desc *desc, scion_stream stream,
                                             scion_bvh *out);

/* Host copies of a BVH's packed device buffers: the node array, the second
 * node array (own-box SoA) and the leaf primitive buffer (48-byte direct
 * triangles or 4-byte ids). Any destination may be NULL (then only its size
 * is reported); sizes[0..2] receive the three byte counts. INVALID_ARG if a
 * given destination is smaller than its buffer. Synchronous (device to
 * host copies on the legacy default stream). */
scion_status scion_debug_bvh_bytes(scion_bvh bvh, void *nodes, uint64_t nodes_cap, void *nodes2, uint64_t nodes2_cap,
                                   void *prims, uint64_t prims_cap, uint64_t *sizes);

/* Records `device` as the GPU the BVH lives on (test hook; nothing is moved):
 * with it a test on one GPU can check that calls reject a BVH from another
 * device with SCION_ERR_INVALID_ARG before anything is issued. The BVH must
 * be given its real device back before it is traced or destroyed. Touches no
 * GPU. */
scion_status scion_debug_set_bvh_device(scion_bvh bvh, int device);

/* Message of the last failing call on the calling host thread (kept per
 * thread; valid until that thread's next failing call). */
const char *scion_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
