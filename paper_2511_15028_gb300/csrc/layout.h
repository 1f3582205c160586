// Physical node and primitive formats shared by the host packer and the
// device traversal. Host and device both include this file.
//
// Two node families implement the paper's logical BVH ADT (Fig. 4:
// Interior(left, right) | Leaf(nprims, data), each with bounds):
//
//  * Own-box binary node ("pbrt", Fig. 4a/4b, Table 1: 32 B). The node holds
//    its own f32 box, a 32-bit reference, a 16-bit primitive count (0 =
//    interior: the split on nprims of Fig. 4b) and the split axis.
//      AoS: one array of 32-byte nodes.
//      SoA: two arrays, boxes (24 B) and references (8 B) ("pbrt-soaos").
//      child_ref direct  : left = I + 1, right = I + ref (DFS pre-order,
//                          build c_o = R - this of Fig. 7).
//      child_ref indirect: left = ref, right = ref + 1 (siblings contiguous).
//      leaf              : prims [ref, ref + count).
//
//  * Quantised own-box binary node (the world-frame bvh2 codecs of Table 1,
//    Section 9.2.5 and App. D.1/D.3): the same tree with the node's box stored
//    as integer codes on one grid spanning the (padded) root box, and one u32
//    word: bits 0-3 primitive count (0 = interior); interior: bits 4-5 split
//    axis, bits 6-31 right offset (direct) or left index (indirect); leaf:
//    bits 4-31 first prim. Limits: leaf_max <= 15, nodes < 2^26.
//      q16  ("sg-pbrt-q16"): 6 x u16 codes (lo.xyz, hi.xyz) + word = 16 B;
//           coordinate = fma(code, step[a], wlo[a]) (one rounding).
//           SoA ("-soaos"): 12 B code array (16 B with align 16) + u32 words.
//      (the shared-slab node of Section 8.3 is a third own-box-like binary
//      node: see kSlabNodeBytes below)
//      eq10 ("sg-eq"): u32 lo codes (x << 20 | y << 10 | z, counted up from
//           wlo), u32 hi codes (same packing, counted down from whi), word =
//           12 B (16 B with align 16); lo = rd(code * bin + wlo),
//           hi = ru(whi - code * bin), each one fused multiply-add rounded
//           outward (App. D.1 rounds the product and the sum separately;
//           the fused form is one instruction and never looser).
//
//  * Children-in-parent wide node (width W = 2, 4, 8; the 8-ary layouts of
//    Table 1, App. D.2). It holds the W child boxes and W child references:
//      [header (u8 only, 16 B)] [boxes] [references], padded to 32 B.
//      header : float3 origin (merged parent box, guard-expanded), 3 exponent
//               bytes (biased by 127) and one spare byte (u8 and u16 codes:
//               coordinate = fma(code, 2^e, origin); the u16 form is the
//               paper's bvh8-q16, App. D.2 with 16-bit codes).
//      boxes  : 6 coordinates per child (lo.xyz, hi.xyz) of 4/2/1 bytes;
//               AoS = per child, SoA = per coordinate across children.
//      refs direct   : u32 per child (bit-stolen, App. D.2 "-ci" reading):
//                      0xFFFFFFFF empty; bit0 = 1 interior, node = ref >> 1;
//                      bit0 = 0 leaf, count = ((ref >> 1) & 15) + 1,
//                      first prim = ref >> 5.
//      refs indirect : u32 base_node, u32 base_prim, u8 meta per child:
//                      0 empty; 0x80 | j interior, node = base_node + j;
//                      1..16 leaf with that many prims; the leaves' prims are
//                      contiguous from base_prim in slot order.
//
//  Primitive buffers:
//    direct  : 48 B per leaf entry: float4 {p0, id}, float4 {p1, 0},
//              float4 {p2, 0} (id stored as the float's bits).
//    indirect: u32 triangle id per leaf entry; vertices in a float4 table
//              and, for indexed meshes, a u32[3] index table.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define SCION_HD __host__ __device__ __forceinline__
#else
#define SCION_HD inline
#endif

namespace scion {

enum BoxPrec : uint32_t {
  PREC_F32 = 0, PREC_F16 = 1, PREC_U8 = 2, PREC_Q16 = 3, PREC_EQ10 = 4, PREC_U16 = 5, PREC_SLAB = 6
};
enum { LAYOUT_AOS = 0, LAYOUT_SOA = 1 };
enum { REF_DIRECT = 0, REF_INDIRECT = 1 };
enum { ORDER_DFS = 0, ORDER_BFS = 1, ORDER_TREELET = 2 };

constexpr uint32_t kEmptyRef = 0xFFFFFFFFu;
constexpr uint32_t kMaxLeaf = 16;
constexpr uint32_t kMaxPrims = 1u << 27;   // direct leaf refs keep 27 offset bits
constexpr uint32_t kMaxNodes = 1u << 30;

// ---- direct child references (wide node)
SCION_HD uint32_t ref_interior(uint32_t node) { return (node << 1) | 1u; }
SCION_HD uint32_t ref_leaf(uint32_t first, uint32_t count) {
  return (first << 5) | ((count - 1u) << 1);
}
SCION_HD bool ref_is_interior(uint32_t r) { return (r & 1u) != 0u; }
SCION_HD uint32_t ref_node(uint32_t r) { return r >> 1; }
SCION_HD uint32_t ref_leaf_first(uint32_t r) { return r >> 5; }
SCION_HD uint32_t ref_leaf_count(uint32_t r) { return ((r >> 1) & 15u) + 1u; }

// ---- indirect meta byte
constexpr uint32_t kMetaInterior = 0x80u;

// ---- wide node geometry
// wide-node box element bytes: f32 4, f16 2, u8 1, u16 2
SCION_HD uint32_t prec_bytes(uint32_t prec) { return prec == PREC_F32 ? 4u : (prec == PREC_U8 ? 1u : 2u); }
// u8 / u16 codes are relative to a frame in the node header
SCION_HD bool prec_is_parent_grid(uint32_t prec) { return prec == PREC_U8 || prec == PREC_U16; }
SCION_HD uint32_t wide_header_bytes(uint32_t prec) { return prec_is_parent_grid(prec) ? 16u : 0u; }
SCION_HD uint32_t wide_box_bytes(uint32_t W, uint32_t prec) { return W * 6u * prec_bytes(prec); }
SCION_HD uint32_t wide_ref_bytes(uint32_t W, uint32_t cref) { return cref == REF_DIRECT ? 4u * W : 8u + W; }
SCION_HD uint32_t wide_ref_offset(uint32_t W, uint32_t prec) {
  return wide_header_bytes(prec) + wide_box_bytes(W, prec);
}
SCION_HD uint32_t wide_node_bytes(uint32_t W, uint32_t prec, uint32_t cref) {
  return wide_ref_offset(W, prec) + wide_ref_bytes(W, cref);
}
SCION_HD uint32_t wide_node_stride(uint32_t W, uint32_t prec, uint32_t cref) {
  return (wide_node_bytes(W, prec, cref) + 31u) & ~31u;
}
// byte offset of coordinate c (0..5 = lo.x lo.y lo.z hi.x hi.y hi.z) of child k
SCION_HD uint32_t wide_box_offset(uint32_t W, uint32_t prec, uint32_t soa, uint32_t k, uint32_t c) {
  uint32_t e = prec_bytes(prec);
  uint32_t idx = soa ? (c * W + k) : (k * 6u + c);
  return wide_header_bytes(prec) + idx * e;
}

// ---- own-box binary node
constexpr uint32_t kBinNodeBytes = 32;  // AoS node
constexpr uint32_t kBinBoxBytes = 24;   // SoA box array element
constexpr uint32_t kBinRefBytes = 8;    // SoA ref array element
// AoS word layout (8 x u32): lo.xyz, hi.xyz, ref, count | axis << 16
SCION_HD uint32_t bin_pack_meta(uint32_t count, uint32_t axis) { return (count & 0xFFFFu) | (axis << 16); }
SCION_HD uint32_t bin_meta_count(uint32_t m) { return m & 0xFFFFu; }
SCION_HD uint32_t bin_meta_axis(uint32_t m) { return (m >> 16) & 3u; }

// ---- quantised own-box binary node (q16 / eq10)
constexpr uint32_t kQBoxBytes = 12;       // 6 x u16, or 2 x u32 + word (eq10 AoS)
constexpr uint32_t kQMaxLeaf = 15;
constexpr uint32_t kQMaxNodes = 1u << 26;
constexpr uint32_t kQ16Max = 65535u, kEq10Max = 1023u;
SCION_HD uint32_t qbin_leaf(uint32_t first, uint32_t count) { return (first << 4) | count; }
SCION_HD uint32_t qbin_interior(uint32_t field, uint32_t axis) { return (field << 6) | (axis << 4); }
SCION_HD uint32_t qbin_count(uint32_t w) { return w & 15u; }
SCION_HD uint32_t qbin_axis(uint32_t w) { return (w >> 4) & 3u; }
SCION_HD uint32_t qbin_field(uint32_t w) { return w >> 6; }
SCION_HD uint32_t qbin_first(uint32_t w) { return w >> 4; }
SCION_HD uint32_t eq10_pack(uint32_t x, uint32_t y, uint32_t z) { return (x << 20) | (y << 10) | z; }
SCION_HD uint32_t eq10_code(uint32_t w, int axis) { return (w >> (20 - 10 * axis)) & 1023u; }
SCION_HD bool prec_is_world_grid(uint32_t prec) { return prec == PREC_Q16 || prec == PREC_EQ10; }
// layouts whose traversal takes per-BVH constants (frame) as launch arguments
SCION_HD bool prec_has_frame(uint32_t prec) { return prec_is_world_grid(prec) || prec == PREC_SLAB; }

// ---- shared-slab binary node (Section 8.3, tree-carried bounds)
// 16 B: f32 slo, f32 shi, u32 field, u32 meta (bin_pack_meta: count | axis << 16).
// Interior: the left child's box is the node's carried box with hi[axis] =
// slo, the right child's with lo[axis] = shi; the root's carried box is the
// frame (padded root box). field: right offset (direct) or left index
// (indirect); leaf: first prim.
constexpr uint32_t kSlabNodeBytes = 16;

constexpr uint32_t kPrimDirectBytes = 48;

// scratch words per BVH (device): work counter, exit counter, status, spare
constexpr uint32_t kScratchWords = 4;

}  // namespace scion
