// Host-side BVH construction and packing. See builder.h.
#include "builder.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>
#include <queue>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace scion {

// ------------------------------------------------------------ descriptor
scion_status normalize_desc(const scion_layout_desc &in, scion_layout_desc *out, bool *own_box) {
  scion_layout_desc d = in;
  if (d.align != 0 && d.align != 16) return SCION_ERR_INVALID_ARG;
  if (d.width != 2 && d.width != 4 && d.width != 8) return SCION_ERR_UNSUPPORTED_LAYOUT;
  if (d.box_layout > 1 || d.box_prec > PREC_SLAB || d.child_ref > 1 || d.prim_ref > 1 || d.order > 2)
    return SCION_ERR_UNSUPPORTED_LAYOUT;
  if (d.leaf_max == 0) d.leaf_max = 4;
  if (d.leaf_max > kMaxLeaf) return SCION_ERR_UNSUPPORTED_LAYOUT;
  if (d.sah_bins == 0) d.sah_bins = 16;
  if (d.sah_bins < 2 || d.sah_bins > 64) return SCION_ERR_UNSUPPORTED_LAYOUT;
  if (d.treelet_bytes == 0) d.treelet_bytes = 1024;
  if (prec_is_world_grid(d.box_prec)) {
    if (d.width != 2 || d.leaf_max > kQMaxLeaf) return SCION_ERR_UNSUPPORTED_LAYOUT;
    if (d.box_prec == PREC_EQ10 && d.box_layout == LAYOUT_SOA) return SCION_ERR_UNSUPPORTED_LAYOUT;
  }
  if (d.box_prec == PREC_SLAB && (d.width != 2 || d.box_layout != LAYOUT_AOS)) return SCION_ERR_UNSUPPORTED_LAYOUT;
  const bool ob = d.width == 2 && (d.box_prec == PREC_F32 || prec_is_world_grid(d.box_prec) ||
                                   d.box_prec == PREC_SLAB);
  if (ob && d.child_ref == REF_DIRECT && d.order != ORDER_DFS) return SCION_ERR_UNSUPPORTED_LAYOUT;
  *out = d;
  *own_box = ob;
  return SCION_OK;
}

// ------------------------------------------------------------ SAH BVH2
namespace {

// Per-triangle record moved by the partitions, so every pass over a node's
// range reads memory sequentially.
struct PrimInfo {
  float lo[3], hi[3], c[3];
  uint32_t id;
};

inline void box_empty(Box3 &b) {
  for (int a = 0; a < 3; ++a) { b.lo[a] = INFINITY; b.hi[a] = -INFINITY; }
}
inline void box_grow(Box3 &b, const float *lo, const float *hi) {
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = std::min(b.lo[a], lo[a]);
    b.hi[a] = std::max(b.hi[a], hi[a]);
  }
}
inline void box_merge(Box3 &b, const Box3 &c) { box_grow(b, c.lo, c.hi); }
// surface area in double: float products overflow for coordinates > ~1e19
inline double box_area(const Box3 &b) {
  double e0 = std::max(0.0, (double)b.hi[0] - (double)b.lo[0]);
  double e1 = std::max(0.0, (double)b.hi[1] - (double)b.lo[1]);
  double e2 = std::max(0.0, (double)b.hi[2] - (double)b.lo[2]);
  return 2.0 * (e0 * e1 + e1 * e2 + e2 * e0);
}

constexpr int kMaxBins = 64;

struct Bins {
  uint32_t cnt[3][kMaxBins];
  Box3 box[3][kMaxBins];
  void clear(int nb) {
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < nb; ++k) { cnt[a][k] = 0; box_empty(box[a][k]); }
  }
};

class SahBuilder {
 public:
  SahBuilder(std::vector<PrimInfo> &recs, uint32_t bins, uint32_t leaf_max, LogicalBVH *out)
      : recs_(recs), bins_((int)bins), leaf_max_(leaf_max), out_(out) {}

  void run() {
    const uint32_t n = (uint32_t)recs_.size();
    out_->nodes.assign(n ? 2 * (size_t)n - 1 : 0, LNode{});
    next_ = 0;
    if (n == 0) {
      out_->prims.clear();
      return;
    }
    tmp_.resize(n);
    struct Task { uint32_t id, first, count; };
    std::vector<Task> big{{alloc(), 0, n}}, small;
    const uint32_t kSerial = 1u << 15;
    while (!big.empty()) {
      Task t = big.back();
      big.pop_back();
      uint32_t l, r, mid;
      if (!split_node(t.id, t.first, t.count, true, &l, &r, &mid)) continue;
      Task lt{l, t.first, mid - t.first}, rt{r, mid, t.first + t.count - mid};
      (lt.count > kSerial ? big : small).push_back(lt);
      (rt.count > kSerial ? big : small).push_back(rt);
    }
    std::sort(small.begin(), small.end(), [](const Task &a, const Task &b) { return a.count > b.count; });
    const long ns = (long)small.size();
#pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < ns; ++i) build_serial(small[i].id, small[i].first, small[i].count);
    out_->nodes.resize(next_.load());
    out_->prims.resize(n);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n; ++i) out_->prims[i] = recs_[i].id;
  }

 private:
  uint32_t alloc() { return next_.fetch_add(1); }

  static int threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
  }
  static int thread_id() {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
  }

  void bounds(uint32_t first, uint32_t count, bool par, Box3 *nb, Box3 *cb) {
    box_empty(*nb);
    box_empty(*cb);
    const PrimInfo *q = recs_.data();
    if (par && count > 4096) {
#pragma omp parallel
      {
        Box3 ln, lc;  // thread-local: no shared cache lines in the loop
        box_empty(ln);
        box_empty(lc);
#pragma omp for schedule(static) nowait
        for (long i = first; i < (long)(first + count); ++i) {
          box_grow(ln, q[i].lo, q[i].hi);
          box_grow(lc, q[i].c, q[i].c);
        }
#pragma omp critical(scion_bounds_merge)
        {
          box_merge(*nb, ln);
          box_merge(*cb, lc);
        }
      }
      return;
    }
    for (uint32_t i = first; i < first + count; ++i) {
      box_grow(*nb, q[i].lo, q[i].hi);
      box_grow(*cb, q[i].c, q[i].c);
    }
  }

  inline int bin_of(const PrimInfo &q, int a, const Box3 &cb, float scale) const {
    int k = (int)((q.c[a] - cb.lo[a]) * scale);
    return std::min(std::max(k, 0), bins_ - 1);
  }

  void bin(uint32_t first, uint32_t count, const Box3 &cb, const float *scale, bool par, Bins *bn) {
    bn->clear(bins_);
    const PrimInfo *q = recs_.data();
    if (par && count > 4096) {
#pragma omp parallel
      {
        Bins b;  // thread-local
        b.clear(bins_);
#pragma omp for schedule(static) nowait
        for (long i = first; i < (long)(first + count); ++i) {
          for (int a = 0; a < 3; ++a) {
            if (!(scale[a] > 0.f)) continue;
            int k = bin_of(q[i], a, cb, scale[a]);
            b.cnt[a][k]++;
            box_grow(b.box[a][k], q[i].lo, q[i].hi);
          }
        }
#pragma omp critical(scion_bins_merge)
        for (int a = 0; a < 3; ++a)
          for (int k = 0; k < bins_; ++k) {
            bn->cnt[a][k] += b.cnt[a][k];
            box_merge(bn->box[a][k], b.box[a][k]);
          }
      }
      return;
    }
    for (uint32_t i = first; i < first + count; ++i) {
      for (int a = 0; a < 3; ++a) {
        if (!(scale[a] > 0.f)) continue;
        int k = bin_of(q[i], a, cb, scale[a]);
        bn->cnt[a][k]++;
        box_grow(bn->box[a][k], q[i].lo, q[i].hi);
      }
    }
  }

  // Stable two-way partition of a large range through the scratch buffer:
  // per-chunk counts, prefix sums, parallel scatter, parallel copy back.
  uint32_t par_partition(uint32_t first, uint32_t count, int axis, int split, const Box3 &cb, float scale) {
    const int nt = threads();
    const uint32_t nch = (uint32_t)nt * 4;
    const uint32_t per = (count + nch - 1) / nch;
    std::vector<uint32_t> nl(nch, 0), nr(nch, 0);
    PrimInfo *q = recs_.data();
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)nch; ++c) {
      const uint32_t b = first + (uint32_t)c * per, e = std::min(first + count, b + per);
      uint32_t l = 0;
      for (uint32_t i = b; i < e; ++i) l += bin_of(q[i], axis, cb, scale) <= split;
      nl[c] = l;
      nr[c] = e > b ? (e - b) - l : 0;
    }
    std::vector<uint32_t> ol(nch), orr(nch);
    uint32_t accl = 0;
    for (uint32_t c = 0; c < nch; ++c) { ol[c] = accl; accl += nl[c]; }
    uint32_t accr = accl;
    for (uint32_t c = 0; c < nch; ++c) { orr[c] = accr; accr += nr[c]; }
    PrimInfo *t = tmp_.data();
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)nch; ++c) {
      const uint32_t b = first + (uint32_t)c * per, e = std::min(first + count, b + per);
      uint32_t pl = first + ol[c], pr = first + orr[c];
      for (uint32_t i = b; i < e; ++i) {
        if (bin_of(q[i], axis, cb, scale) <= split) t[pl++] = q[i];
        else t[pr++] = q[i];
      }
    }
#pragma omp parallel for schedule(static)
    for (long i = first; i < (long)(first + count); ++i) q[i] = t[i];
    return first + accl;
  }

  // Decide leaf or split for node `id`; on a split allocate the children and
  // partition the range. Returns false for a leaf.
  bool split_node(uint32_t id, uint32_t first, uint32_t count, bool par, uint32_t *l,
                  uint32_t *r, uint32_t *mid_out) {
    LNode &nd = out_->nodes[id];
    Box3 nb, cb;
    bounds(first, count, par, &nb, &cb);
    nd.box = nb;
    float scale[3];
    for (int a = 0; a < 3; ++a) {
      float e = cb.hi[a] - cb.lo[a];
      scale[a] = e > 0.f ? (float)bins_ / e : 0.f;
    }
    int best_axis = -1, best_bin = -1;
    double best_cost = INFINITY;
    if (count > 1) {
      Bins bn;
      bin(first, count, cb, scale, par, &bn);
      for (int a = 0; a < 3; ++a) {
        if (!(scale[a] > 0.f)) continue;
        double rarea[kMaxBins];
        uint32_t rcnt[kMaxBins];
        Box3 acc;
        box_empty(acc);
        uint32_t n = 0;
        for (int k = bins_ - 1; k > 0; --k) {
          box_merge(acc, bn.box[a][k]);
          n += bn.cnt[a][k];
          rarea[k] = box_area(acc);
          rcnt[k] = n;
        }
        box_empty(acc);
        n = 0;
        for (int k = 0; k < bins_ - 1; ++k) {
          box_merge(acc, bn.box[a][k]);
          n += bn.cnt[a][k];
          if (n == 0 || rcnt[k + 1] == 0) continue;
          double c = box_area(acc) * (double)n + rarea[k + 1] * (double)rcnt[k + 1];
          if (c < best_cost) { best_cost = c; best_axis = a; best_bin = k; }
        }
      }
    }
    const double area = box_area(nb);
    const double leaf_cost = area * (double)count;
    const double split_cost = area + best_cost;
    if (count == 1 || (count <= leaf_max_ && (best_axis < 0 || leaf_cost <= split_cost))) {
      nd.first = first;
      nd.count = count;
      nd.left = nd.right = 0;
      nd.axis = 0;
      return false;
    }
    PrimInfo *q = recs_.data();
    uint32_t mid;
    int axis = best_axis;
    if (best_axis < 0) {
      mid = first + count / 2;
      float ext = -1.f;
      for (int a = 0; a < 3; ++a)
        if (nb.hi[a] - nb.lo[a] > ext) { ext = nb.hi[a] - nb.lo[a]; axis = a; }
    } else {
      const float sc = scale[best_axis];
      if (par && count > (1u << 18)) {
        mid = par_partition(first, count, best_axis, best_bin, cb, sc);
      } else {
        PrimInfo *m = std::partition(q + first, q + first + count, [&](const PrimInfo &x) {
          return bin_of(x, best_axis, cb, sc) <= best_bin;
        });
        mid = (uint32_t)(m - q);
      }
      if (mid == first || mid == first + count) mid = first + count / 2;
    }
    nd.count = 0;
    nd.first = 0;
    nd.axis = (uint32_t)std::max(axis, 0);
    nd.left = alloc();
    nd.right = alloc();
    *l = nd.left;
    *r = nd.right;
    *mid_out = mid;
    return true;
  }

  void build_serial(uint32_t id, uint32_t first, uint32_t count) {
    uint32_t l, r, mid;
    if (!split_node(id, first, count, false, &l, &r, &mid)) return;
    build_serial(l, first, mid - first);
    build_serial(r, mid, first + count - mid);
  }

  std::vector<PrimInfo> &recs_;
  std::vector<PrimInfo> tmp_;
  int bins_;
  uint32_t leaf_max_;
  LogicalBVH *out_;
  std::atomic<uint32_t> next_{0};
};

inline bool finite_tri(const float *v0, const float *v1, const float *v2) {
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(v0[k]) || !std::isfinite(v1[k]) || !std::isfinite(v2[k])) return false;
  return true;
}

inline void tri_verts(const BuildInput &in, uint64_t t, const float **v0, const float **v1,
                      const float **v2) {
  if (in.indices) {
    *v0 = in.verts + 3 * (uint64_t)in.indices[3 * t];
    *v1 = in.verts + 3 * (uint64_t)in.indices[3 * t + 1];
    *v2 = in.verts + 3 * (uint64_t)in.indices[3 * t + 2];
  } else {
    *v0 = in.verts + 9 * t;
    *v1 = in.verts + 9 * t + 3;
    *v2 = in.verts + 9 * t + 6;
  }
}

}  // namespace

void build_logical(const BuildInput &in, uint32_t bins, uint32_t leaf_max, LogicalBVH *out) {
  const uint64_t n = in.n_tris;
  std::vector<uint8_t> ok(n);
#pragma omp parallel for schedule(static)
  for (long long t = 0; t < (long long)n; ++t) {
    const float *v0, *v1, *v2;
    tri_verts(in, (uint64_t)t, &v0, &v1, &v2);
    ok[t] = finite_tri(v0, v1, v2);
  }
  // records of the finite triangles, in id order
  std::vector<uint32_t> pos(n + 1, 0);
  for (uint64_t t = 0; t < n; ++t) pos[t + 1] = pos[t] + ok[t];
  std::vector<PrimInfo> recs(pos[n]);
#pragma omp parallel for schedule(static)
  for (long long t = 0; t < (long long)n; ++t) {
    if (!ok[t]) continue;
    const float *v0, *v1, *v2;
    tri_verts(in, (uint64_t)t, &v0, &v1, &v2);
    PrimInfo &q = recs[pos[t]];
    for (int a = 0; a < 3; ++a) {
      q.lo[a] = std::min(v0[a], std::min(v1[a], v2[a]));
      q.hi[a] = std::max(v0[a], std::max(v1[a], v2[a]));
      q.c[a] = (v0[a] + v1[a] + v2[a]) * (1.0f / 3.0f);
    }
    q.id = (uint32_t)t;
  }
  SahBuilder b(recs, bins, leaf_max, out);
  b.run();
}

// ------------------------------------------------------------ node orders
namespace {

// Abstract tree of physical nodes in CSR form: the physical-node children of
// node i (in slot order) are kid[off[i] .. off[i+1]); area[i] is its surface
// area. Node 0 is the root.
struct OrderTree {
  std::vector<uint32_t> off, kid;
  std::vector<float> area;
  size_t size() const { return area.size(); }
  uint32_t nk(uint32_t i) const { return off[i + 1] - off[i]; }
  const uint32_t *kids(uint32_t i) const { return kid.data() + off[i]; }
};

std::vector<uint32_t> order_nodes(const OrderTree &t, uint32_t order, bool group_siblings,
                                  uint32_t stride, uint32_t treelet_bytes) {
  const size_t n = t.size();
  std::vector<uint32_t> out;
  out.reserve(n);
  if (n == 0) return out;
  if (order == ORDER_BFS) {
    out.push_back(0);
    for (size_t h = 0; h < out.size(); ++h) {
      const uint32_t x = out[h];
      for (uint32_t k = 0; k < t.nk(x); ++k) out.push_back(t.kids(x)[k]);
    }
    return out;
  }
  if (order == ORDER_DFS) {
    std::vector<uint32_t> st{0};
    if (!group_siblings) {
      while (!st.empty()) {
        const uint32_t x = st.back();
        st.pop_back();
        out.push_back(x);
        for (uint32_t k = t.nk(x); k-- > 0;) st.push_back(t.kids(x)[k]);
      }
    } else {
      out.push_back(0);
      while (!st.empty()) {
        const uint32_t x = st.back();
        st.pop_back();
        for (uint32_t k = 0; k < t.nk(x); ++k) out.push_back(t.kids(x)[k]);
        for (uint32_t k = t.nk(x); k-- > 0;) st.push_back(t.kids(x)[k]);
      }
    }
    return out;
  }
  // Treelets: grow a cluster from a root by repeatedly adding the frontier
  // node (or sibling group) of largest surface area while the cluster fits the
  // byte budget; what is left on the frontier seeds later clusters.
  using Item = std::pair<float, uint32_t>;
  std::vector<Item> heap, rest;
  auto push = [&](Item it) { heap.push_back(it); std::push_heap(heap.begin(), heap.end()); };
  auto pop = [&]() { std::pop_heap(heap.begin(), heap.end()); Item it = heap.back(); heap.pop_back(); return it; };
  std::deque<uint32_t> roots;
  if (!group_siblings) {
    roots.push_back(0);
    while (!roots.empty()) {
      const uint32_t r = roots.front();
      roots.pop_front();
      heap.clear();
      out.push_back(r);
      uint32_t bytes = stride;
      for (uint32_t k = 0; k < t.nk(r); ++k) push({t.area[t.kids(r)[k]], t.kids(r)[k]});
      while (!heap.empty() && bytes + stride <= treelet_bytes) {
        const uint32_t c = pop().second;
        out.push_back(c);
        bytes += stride;
        for (uint32_t k = 0; k < t.nk(c); ++k) push({t.area[t.kids(c)[k]], t.kids(c)[k]});
      }
      rest.clear();
      while (!heap.empty()) rest.push_back(pop());
      for (auto &it : rest) roots.push_back(it.second);
    }
    return out;
  }
  // sibling groups, identified by their parent node
  out.push_back(0);
  if (t.nk(0) > 0) roots.push_back(0);
  while (!roots.empty()) {
    const uint32_t gp = roots.front();
    roots.pop_front();
    heap.clear();
    uint32_t bytes = 0;
    auto emit = [&](uint32_t parent) {
      for (uint32_t k = 0; k < t.nk(parent); ++k) out.push_back(t.kids(parent)[k]);
      bytes += stride * t.nk(parent);
      for (uint32_t k = 0; k < t.nk(parent); ++k) {
        const uint32_t c = t.kids(parent)[k];
        if (t.nk(c) > 0) push({t.area[c], c});
      }
    };
    emit(gp);
    while (!heap.empty()) {
      const uint32_t c = heap.front().second;
      if (bytes + stride * t.nk(c) > treelet_bytes) break;
      pop();
      emit(c);
    }
    rest.clear();
    while (!heap.empty()) rest.push_back(pop());
    for (auto &it : rest) roots.push_back(it.second);
  }
  return out;
}

float area_of(const Box3 &b) { return (float)box_area(b); }

// Leaf entries [at, at + count) of a logical leaf, in the leaf's order.
void emit_prims(const BuildInput &in, const LogicalBVH &lb, const LNode &leaf, HostBVH *out, uint32_t at) {
  for (uint32_t k = 0; k < leaf.count; ++k) {
    const uint32_t id = lb.prims[leaf.first + k];
    if (out->desc.prim_ref == REF_DIRECT) {
      const float *v0, *v1, *v2;
      tri_verts(in, id, &v0, &v1, &v2);
      float *rec = out->prim_direct.data() + 12 * (size_t)(at + k);
      rec[0] = v0[0]; rec[1] = v0[1]; rec[2] = v0[2];
      std::memcpy(&rec[3], &id, 4);
      rec[4] = v1[0]; rec[5] = v1[1]; rec[6] = v1[2]; rec[7] = 0.f;
      rec[8] = v2[0]; rec[9] = v2[1]; rec[10] = v2[2]; rec[11] = 0.f;
    } else {
      out->prim_ids[at + k] = id;
    }
  }
}

// Exclusive prefix sum in place; returns the total.
uint64_t exclusive_scan(std::vector<uint32_t> &v) {
  uint64_t acc = 0;
  for (auto &x : v) {
    const uint32_t c = x;
    x = (uint32_t)acc;
    acc += c;
  }
  return acc;
}

void alloc_prims(HostBVH *out, uint64_t entries) {
  out->n_leaf_entries = (uint32_t)entries;
  if (out->desc.prim_ref == REF_DIRECT) out->prim_direct.assign(12 * entries, 0.f);
  else out->prim_ids.assign(entries, 0u);
}

// Stored-tree depth: parents come before children in every order.
uint32_t tree_depth(const OrderTree &t, const std::vector<uint32_t> &ord) {
  std::vector<uint32_t> depth(t.size(), 1);
  uint32_t maxd = 1;
  for (uint32_t x : ord)
    for (uint32_t k = 0; k < t.nk(x); ++k) {
      depth[t.kids(x)[k]] = depth[x] + 1;
      maxd = std::max(maxd, depth[x] + 1);
    }
  return maxd;
}

}  // namespace

// ------------------------------------------------------------ packing
// Count pass (node order, leaf-entry offsets by prefix sum, one allocation per
// buffer), then a parallel fill pass (App. F: rec_count, allocate, rec_build).
scion_status pack_bvh(const BuildInput &in, const LogicalBVH &lb, const scion_layout_desc &desc,
                      bool own_box, HostBVH *out, std::string *err) {
  out->desc = desc;
  out->own_box = own_box;
  out->n_tris = (uint32_t)in.n_tris;
  out->n_verts = (uint32_t)in.n_verts;
  out->indexed = in.indices != nullptr;
  out->n_leaf_entries = 0;
  // vertex / index tables (used by indirect prims and by the backward pass)
  out->verts4.assign(4 * (size_t)in.n_verts, 0.f);
#pragma omp parallel for schedule(static)
  for (long long v = 0; v < (long long)in.n_verts; ++v)
    for (int k = 0; k < 3; ++k) out->verts4[4 * v + k] = in.verts[3 * v + k];
  if (in.indices) out->indices.assign(in.indices, in.indices + 3 * in.n_tris);
  const uint32_t W = desc.width;
  const size_t nl = lb.nodes.size();
  if (nl == 0) {  // no hittable triangle
    out->n_nodes = 0;
    out->root_ref = kEmptyRef;
    out->depth = 0;
    out->stack_need = 0;
    return SCION_OK;
  }

  if (own_box) {
    // ---- own-box binary nodes: every logical node is a physical node
    OrderTree t;
    t.off.assign(nl + 1, 0);
    t.area.resize(nl);
    for (size_t i = 0; i < nl; ++i) t.off[i + 1] = t.off[i] + (lb.nodes[i].count == 0 ? 2u : 0u);
    t.kid.resize(t.off[nl]);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)nl; ++i) {
      t.area[i] = area_of(lb.nodes[i].box);
      if (lb.nodes[i].count == 0) {
        t.kid[t.off[i]] = lb.nodes[i].left;
        t.kid[t.off[i] + 1] = lb.nodes[i].right;
      }
    }
    const bool group = desc.child_ref == REF_INDIRECT;
    std::vector<uint32_t> ord = order_nodes(t, desc.order, group, kBinNodeBytes, desc.treelet_bytes);
    std::vector<uint32_t> phys(nl);
    for (size_t i = 0; i < ord.size(); ++i) phys[ord[i]] = (uint32_t)i;
    // count pass: leaf entries per physical node, prefix-summed
    std::vector<uint32_t> pbase(nl);
    for (size_t pi = 0; pi < nl; ++pi) pbase[pi] = lb.nodes[ord[pi]].count;
    alloc_prims(out, exclusive_scan(pbase));
    out->n_nodes = (uint32_t)nl;
    const uint32_t prec = desc.box_prec;
    const bool soa = desc.box_layout == LAYOUT_SOA, a16 = desc.align == 16;
    const bool quant = prec_is_world_grid(prec);
    if (quant && nl >= kQMaxNodes) {
      *err = "too many nodes for the quantised own-box node";
      return SCION_ERR_UNSUPPORTED_LAYOUT;
    }
    uint32_t ref_bytes = 0;  // SoA word/ref array element
    if (prec == PREC_SLAB) {
      out->node_stride = kSlabNodeBytes;
    } else if (!quant) {
      out->node_stride = soa ? (a16 ? 32u : kBinBoxBytes) : kBinNodeBytes;
      ref_bytes = soa ? kBinRefBytes : 0u;
    } else if (prec == PREC_Q16) {
      out->node_stride = soa ? (a16 ? 16u : kQBoxBytes) : 16u;
      ref_bytes = soa ? 4u : 0u;
    } else {
      out->node_stride = a16 ? 16u : kQBoxBytes;
    }
    out->nodes.assign((size_t)nl * out->node_stride, 0);
    if (ref_bytes) out->nodes2.assign((size_t)nl * ref_bytes, 0);
    // world grid over the padded root box: q16 {wlo, step}, eq10 {wlo, whi, bin}
    float bins_inv[3] = {0.f, 0.f, 0.f};
    if (quant) world_frame(prec, padded(lb.nodes[0].box), out->frame, bins_inv);
    // shared slab: the plane axis of each node is the one whose two carried
    // child boxes have the least total surface area (the boxes the traversal
    // tests); carried boxes top-down from the padded root box
    std::vector<uint8_t> slab_axis;
    if (prec == PREC_SLAB) {
      const Box3 root = padded(lb.nodes[0].box);
      for (int a = 0; a < 3; ++a) {
        out->frame[a] = root.lo[a];
        out->frame[3 + a] = root.hi[a];
      }
      slab_axis.assign(nl, 0);
      std::vector<std::pair<uint32_t, Box3>> todo{{0u, root}};
      while (!todo.empty()) {
        const uint32_t x = todo.back().first;
        const Box3 cx = todo.back().second;
        todo.pop_back();
        const LNode &nd = lb.nodes[x];
        if (nd.count > 0) continue;
        const Box3 pl = padded(lb.nodes[nd.left].box), pr = padded(lb.nodes[nd.right].box);
        int best = (int)nd.axis;
        double best_cost = INFINITY;
        Box3 bl = cx, br = cx;
        for (int a = 0; a < 3; ++a) {
          Box3 l = cx, r = cx;
          l.hi[a] = pl.hi[a];
          r.lo[a] = pr.lo[a];
          const double cost = box_area(l) + box_area(r);
          if (cost < best_cost) {
            best_cost = cost;
            best = a;
            bl = l;
            br = r;
          }
        }
        slab_axis[x] = (uint8_t)best;
        todo.push_back({nd.left, bl});
        todo.push_back({nd.right, br});
      }
    }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long long pi = 0; pi < (long long)nl; ++pi) {
      const LNode &nd = lb.nodes[ord[pi]];
      uint32_t ref, meta;
      if (nd.count > 0) {
        ref = pbase[pi];
        meta = bin_pack_meta(nd.count, 0);
        emit_prims(in, lb, nd, out, pbase[pi]);
      } else {
        const uint32_t l = phys[nd.left], r = phys[nd.right];
        if (desc.child_ref == REF_DIRECT) {
          bad |= l != (uint32_t)pi + 1;
          ref = r - (uint32_t)pi;
        } else {
          bad |= r != l + 1;
          ref = l;
        }
        meta = bin_pack_meta(0, nd.axis);
      }
      uint8_t *p = out->nodes.data() + pi * out->node_stride;
      if (prec == PREC_SLAB) {
        if (nd.count == 0) {
          const uint32_t ax = slab_axis[ord[pi]];
          encode_slab_planes(lb.nodes[nd.left].box, lb.nodes[nd.right].box, ax, p);
          meta = bin_pack_meta(0, ax);
        }
        put_u32(p + 8, ref);
        put_u32(p + 12, meta);
        continue;
      }
      bad |= encode_own_box(prec, nd.box, out->frame, bins_inv, p) ? 0 : 2;
      if (!quant) {
        uint8_t *q = soa ? out->nodes2.data() + pi * kBinRefBytes : p + 24;
        put_u32(q, ref);
        put_u32(q + 4, meta);
      } else {
        const uint32_t word = nd.count > 0 ? qbin_leaf(ref, nd.count) : qbin_interior(ref, nd.axis);
        put_u32(prec == PREC_Q16 ? (soa ? out->nodes2.data() + pi * 4 : p + 12) : p + 8, word);
      }
    }
    if (bad & 1) {
      *err = "node order violates the child reference encoding";
      return SCION_ERR_UNSUPPORTED_LAYOUT;
    }
    if (bad & 2) {
      *err = "world-grid enclosure";
      return SCION_ERR_BAD_INPUT;
    }
    out->root_ref = 0;
    out->depth = tree_depth(t, ord);
    out->stack_need = out->depth;
    return SCION_OK;
  }

  // ---- children-in-parent wide nodes: collapse the BVH2 to width W by
  // repeatedly opening the interior child of largest surface area
  std::vector<WNode> wn;
  wn.reserve(nl / 2 + 1);
  std::vector<uint32_t> wide_of(nl, kEmptyRef);
  {
    std::vector<uint32_t> todo{0};
    wide_of[0] = 0;
    wn.push_back(WNode{});
    while (!todo.empty()) {
      const uint32_t li = todo.back();
      todo.pop_back();
      const uint32_t wi = wide_of[li];
      WNode w{};
      w.lnode = li;
      if (lb.nodes[li].count > 0) {
        w.n = 1;  // a leaf root: one-child wide root
        w.child[0] = li;
      } else {
        w.n = 2;
        w.child[0] = lb.nodes[li].left;
        w.child[1] = lb.nodes[li].right;
        while (w.n < W) {
          int best = -1;
          double ba = -1.0;
          for (uint32_t k = 0; k < w.n; ++k) {
            const LNode &c = lb.nodes[w.child[k]];
            if (c.count == 0) {
              const double a = box_area(c.box);
              if (a > ba) { ba = a; best = (int)k; }
            }
          }
          if (best < 0) break;
          const LNode &c = lb.nodes[w.child[best]];
          for (uint32_t k = w.n; k > (uint32_t)best + 1; --k) w.child[k] = w.child[k - 1];
          w.child[best] = c.left;
          w.child[best + 1] = c.right;
          ++w.n;
        }
        for (uint32_t k = 0; k < w.n; ++k) {
          if (lb.nodes[w.child[k]].count == 0) {
            wide_of[w.child[k]] = (uint32_t)wn.size();
            wn.push_back(WNode{});
            todo.push_back(w.child[k]);
          }
        }
      }
      wn[wi] = w;
    }
  }
  const size_t nw = wn.size();
  if (nw >= kMaxNodes) { *err = "too many nodes"; return SCION_ERR_INVALID_ARG; }
  OrderTree t;
  t.off.assign(nw + 1, 0);
  t.area.resize(nw);
  for (size_t i = 0; i < nw; ++i) {
    uint32_t c = 0;
    for (uint32_t k = 0; k < wn[i].n; ++k) c += lb.nodes[wn[i].child[k]].count == 0;
    t.off[i + 1] = t.off[i] + c;
  }
  t.kid.resize(t.off[nw]);
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < (long long)nw; ++i) {
    t.area[i] = area_of(lb.nodes[wn[i].lnode].box);
    uint32_t o = t.off[i];
    for (uint32_t k = 0; k < wn[i].n; ++k)
      if (lb.nodes[wn[i].child[k]].count == 0) t.kid[o++] = wide_of[wn[i].child[k]];
  }
  const uint32_t prec = desc.box_prec, soa = desc.box_layout, cref = desc.child_ref;
  const uint32_t stride = wide_node_stride(W, prec, cref);
  std::vector<uint32_t> ord = order_nodes(t, desc.order, cref == REF_INDIRECT, stride, desc.treelet_bytes);
  std::vector<uint32_t> phys(nw);
  for (size_t i = 0; i < ord.size(); ++i) phys[ord[i]] = (uint32_t)i;
  // count pass: leaf entries per physical node (slot order), prefix-summed
  std::vector<uint32_t> pbase(nw);
  for (size_t pi = 0; pi < nw; ++pi) {
    const WNode &w = wn[ord[pi]];
    uint32_t c = 0;
    for (uint32_t k = 0; k < w.n; ++k) c += lb.nodes[w.child[k]].count;
    pbase[pi] = c;
  }
  alloc_prims(out, exclusive_scan(pbase));
  out->n_nodes = (uint32_t)nw;
  out->node_stride = stride;
  out->nodes.assign((size_t)nw * stride, 0);
  const uint32_t ref_off = wide_ref_offset(W, prec);
  int bad = 0;  // 1: siblings not contiguous, 2: f16 enclosure, 4: u8 enclosure
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
  for (long long pi = 0; pi < (long long)nw; ++pi) {
    const WNode &w = wn[ord[pi]];
    uint8_t *p = out->nodes.data() + (size_t)pi * stride;
    Box3 cb[8];
    for (uint32_t k = 0; k < w.n; ++k) cb[k] = lb.nodes[w.child[k]].box;
    // references and leaf primitives (slot order)
    uint32_t first_interior = kEmptyRef, rank = 0, at = pbase[pi];
    for (uint32_t k = 0; k < W; ++k) {
      uint32_t refv = kEmptyRef, meta = 0;
      if (k < w.n) {
        const LNode &c = lb.nodes[w.child[k]];
        if (c.count == 0) {
          const uint32_t cp = phys[wide_of[w.child[k]]];
          if (first_interior == kEmptyRef) first_interior = cp;
          if (cref == REF_INDIRECT && cp != first_interior + rank) bad |= 1;
          refv = ref_interior(cp);
          meta = kMetaInterior | rank;
          ++rank;
        } else {
          refv = ref_leaf(at, c.count);
          meta = c.count;
          emit_prims(in, lb, c, out, at);
          at += c.count;
        }
      }
      if (cref == REF_DIRECT) put_u32(p + ref_off + 4 * k, refv);
      else p[ref_off + 8 + k] = (uint8_t)meta;
    }
    if (cref == REF_INDIRECT) {
      put_u32(p + ref_off, first_interior == kEmptyRef ? 0u : first_interior);
      put_u32(p + ref_off + 4, pbase[pi]);
    }
    // boxes
    bad |= encode_wide_boxes(W, prec, soa, cb, w.n, p);
  }
  if (bad & 1) { *err = "siblings not contiguous"; return SCION_ERR_UNSUPPORTED_LAYOUT; }
  if (bad & 2) { *err = "f16 enclosure"; return SCION_ERR_BAD_INPUT; }
  if (bad & 4) { *err = "u8/u16 enclosure"; return SCION_ERR_BAD_INPUT; }
  out->root_ref = ref_interior(0);
  out->depth = tree_depth(t, ord);
  out->stack_need = (W - 1) * out->depth + 1;
  return SCION_OK;
}

// ------------------------------------------------------------ decode (round trip)
int decode_node(const HostBVH &b, uint32_t node, DecodedChild *ch, Box3 *own) {
  const scion_layout_desc &d = b.desc;
  if (node >= b.n_nodes) return -1;
  if (b.own_box) {
    const bool soa = d.box_layout == LAYOUT_SOA;
    const uint8_t *p = b.nodes.data() + (size_t)node * b.node_stride;
    uint32_t ref, cnt;
    if (d.box_prec == PREC_SLAB) {
      // the carried box depends on the ancestors: left to the caller
      for (int a = 0; a < 3; ++a) own->lo[a] = own->hi[a] = NAN;
      ref = get_u32(p + 8);
      cnt = bin_meta_count(get_u32(p + 12));
    } else if (d.box_prec == PREC_F32) {
      const uint8_t *q = soa ? b.nodes2.data() + (size_t)node * kBinRefBytes : p + 24;
      for (int a = 0; a < 3; ++a) {
        own->lo[a] = get_f32(p + 4 * a);
        own->hi[a] = get_f32(p + 12 + 4 * a);
      }
      ref = get_u32(q);
      cnt = bin_meta_count(get_u32(q + 4));
    } else {
      uint32_t word;
      if (d.box_prec == PREC_Q16) {
        for (int a = 0; a < 3; ++a) {
          own->lo[a] = q16_decode(get_u16(p + 2 * a), b.frame[3 + a], b.frame[a]);
          own->hi[a] = q16_decode(get_u16(p + 6 + 2 * a), b.frame[3 + a], b.frame[a]);
        }
        word = get_u32(soa ? b.nodes2.data() + (size_t)node * 4 : p + 12);
      } else {
        const uint32_t wl = get_u32(p), wh = get_u32(p + 4);
        for (int a = 0; a < 3; ++a) {
          own->lo[a] = eq10_decode_lo(eq10_code(wl, a), b.frame[6 + a], b.frame[a]);
          own->hi[a] = eq10_decode_hi(eq10_code(wh, a), b.frame[6 + a], b.frame[3 + a]);
        }
        word = get_u32(p + 8);
      }
      cnt = qbin_count(word);
      ref = cnt > 0 ? qbin_first(word) : qbin_field(word);
    }
    if (cnt > 0) {
      ch[0].kind = 2;
      ch[0].first = ref;
      ch[0].count = cnt;
      return 1;
    }
    const uint32_t l = d.child_ref == REF_DIRECT ? node + 1 : ref;
    const uint32_t r = d.child_ref == REF_DIRECT ? node + ref : ref + 1;
    ch[0].kind = 1; ch[0].node = l;
    ch[1].kind = 1; ch[1].node = r;
    return 2;
  }
  const uint32_t W = d.width, prec = d.box_prec, soa = d.box_layout, cref = d.child_ref;
  const uint8_t *p = b.nodes.data() + (size_t)node * b.node_stride;
  const uint32_t ref_off = wide_ref_offset(W, prec);
  uint32_t leaf_acc = 0;
  for (uint32_t k = 0; k < W; ++k) {
    DecodedChild &c = ch[k];
    c.kind = 0;
    if (cref == REF_DIRECT) {
      const uint32_t r = get_u32(p + ref_off + 4 * k);
      if (r == kEmptyRef) continue;
      if (ref_is_interior(r)) { c.kind = 1; c.node = ref_node(r); }
      else { c.kind = 2; c.first = ref_leaf_first(r); c.count = ref_leaf_count(r); }
    } else {
      const uint32_t bn = get_u32(p + ref_off), bp = get_u32(p + ref_off + 4);
      const uint32_t m = p[ref_off + 8 + k];
      if (m == 0) continue;
      if (m & kMetaInterior) { c.kind = 1; c.node = bn + (m & 0x7Fu); }
      else { c.kind = 2; c.first = bp + leaf_acc; c.count = m; leaf_acc += m; }
    }
    for (uint32_t a = 0; a < 3; ++a) {
      const uint32_t olo = wide_box_offset(W, prec, soa, k, a), ohi = wide_box_offset(W, prec, soa, k, 3 + a);
      if (prec == PREC_F32) {
        c.box.lo[a] = get_f32(p + olo);
        c.box.hi[a] = get_f32(p + ohi);
      } else if (prec == PREC_F16) {
        c.box.lo[a] = f16_to_f32(get_u16(p + olo));
        c.box.hi[a] = f16_to_f32(get_u16(p + ohi));
      } else {
        const float origin = get_f32(p + 4 * a);
        uint32_t bits = (uint32_t)p[12 + a] << 23;
        float scale;
        std::memcpy(&scale, &bits, 4);
        const uint32_t ql = prec == PREC_U8 ? p[olo] : get_u16(p + olo);
        const uint32_t qh = prec == PREC_U8 ? p[ohi] : get_u16(p + ohi);
        c.box.lo[a] = u8_decode(ql, scale, origin);
        c.box.hi[a] = u8_decode(qh, scale, origin);
      }
    }
  }
  return (int)W;
}

}  // namespace scion
