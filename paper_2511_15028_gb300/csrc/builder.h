// Host-side BVH construction and packing (C++17, OpenMP).
//
// Two-phase construction (Section 5.1): a logical binned-SAH BVH2 is built
// first (Section 9.1: top-down partitioning guided by SAH over binned
// centroids), then packed into the requested physical layout with the
// count-then-fill pattern of the paper's generated constructor (App. F:
// rec_count sizes every buffer, one allocation per buffer, rec_build fills it).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/scion.h"
#include "codec.h"
#include "layout.h"

namespace scion {

// Logical BVH2 node (the paper's BVH ADT): leaf iff count > 0.
struct LNode {
  Box3 box;
  uint32_t left, right;   // children (interior)
  uint32_t first, count;  // range in LogicalBVH::prims (leaf)
  uint32_t axis;          // split axis (interior)
};

struct LogicalBVH {
  std::vector<LNode> nodes;     // nodes[0] is the root (empty if no triangles)
  std::vector<uint32_t> prims;  // triangle ids, leaves reference ranges
};

// Wide (collapsed) node: children are logical nodes; a child is a leaf iff
// its logical node is a leaf, otherwise it is the wide node wide_of[child].
struct WNode {
  uint32_t lnode;       // logical node whose box this wide node covers
  uint32_t n;           // child count (1..W)
  uint32_t child[8];    // logical node ids
};

struct HostBVH {
  scion_layout_desc desc;
  bool own_box = false;             // width-2 own-box node (f32, q16, eq10)
  uint32_t n_tris = 0, n_verts = 0;
  bool indexed = false;
  std::vector<uint8_t> nodes;       // node buffer (AoS nodes or SoA boxes)
  std::vector<uint8_t> nodes2;      // own-box SoA reference array
  uint32_t node_stride = 0;         // bytes per node in `nodes`
  uint32_t n_nodes = 0;
  std::vector<float> prim_direct;   // 12 floats per leaf entry
  std::vector<uint32_t> prim_ids;   // indirect leaf entries
  uint32_t n_leaf_entries = 0;
  std::vector<float> verts4;        // float4 vertex table
  std::vector<uint32_t> indices;    // u32[3] per triangle (indexed meshes)
  uint32_t root_ref = kEmptyRef;    // wide: encoded ref of the root; own-box: 0
  uint32_t depth = 0;               // levels of the stored tree
  uint32_t stack_need = 0;          // worst-case traversal stack entries
  float frame[9] = {};              // world grid: q16 {wlo, step}, eq10 {wlo, whi, bin}
  double build_ms = 0.0;             // whole host build (logical + pack)
  double logical_ms = 0.0;           // logical BVH2 construction (host wall or GPU device time)
  double pack_ms = 0.0;              // packing into the layout
};

struct BuildInput {
  const float *verts;        // host float[n_verts][3]
  uint64_t n_verts;
  const uint32_t *indices;   // host u32[n_tris][3] or nullptr
  uint64_t n_tris;
};

// Validate a descriptor (fills defaults). Returns SCION_OK or an error code.
scion_status normalize_desc(const scion_layout_desc &in, scion_layout_desc *out, bool *own_box);

// Build the logical BVH2 over finite triangles.
void build_logical(const BuildInput &in, uint32_t bins, uint32_t leaf_max, LogicalBVH *out);

// Pack a logical BVH into the physical layout of `desc` (already normalized).
scion_status pack_bvh(const BuildInput &in, const LogicalBVH &lb, const scion_layout_desc &desc,
                      bool own_box, HostBVH *out, std::string *err);

// Decode one packed node back to its logical view (round-trip check).
struct DecodedChild {
  Box3 box;           // decoded (conservative) box
  int kind;           // 0 empty, 1 interior, 2 leaf
  uint32_t node;      // physical node index (interior)
  uint32_t first, count;  // leaf prim range (leaf)
};
// For a wide node: fills up to W children. For an own-box node: returns the
// node's own box in children[0] and its two children (or leaf) as kind.
int decode_node(const HostBVH &b, uint32_t node, DecodedChild *children, Box3 *own_box);

}  // namespace scion
