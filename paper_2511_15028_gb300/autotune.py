"""Per-scene layout and traversal-parameter autotuner for the batched launch.

The paper's design-space exploration (Section 9.2) finds that the best layout
depends on the scene, the rays and the machine. Here that choice is made per
scene by measurement: the scene is built once as a logical BVH2 and packed into
every candidate layout (scion_build_many); a sample of the scene's own rays is
traced with each (layout, parameters) candidate, timed with CUDA events; the
fastest wins and the choice is cached under the caller's key.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import scion

# Node layouts the batched kernel runs in one launch (direct child
# references): the pbrt bvh2 node and its 16-byte world-grid version, 4-wide
# SoA nodes (f32; f32 and u8 boxes in breadth-first order, which win once the
# BVH is far larger than L2) and 8-wide f16 / u8 nodes.
CANDIDATE_LAYOUTS = {
    "bvh2_aos_f32": dict(width=2, box_layout="aos", box_prec="f32"),
    "bvh2_aos_q16": dict(width=2, box_layout="aos", box_prec="q16"),
    "bvh4_soa_f32": dict(width=4, box_layout="soa", box_prec="f32"),
    "bvh4_soa_f32_bfs": dict(width=4, box_layout="soa", box_prec="f32", order="bfs"),
    "bvh4_soa_u8_bfs": dict(width=4, box_layout="soa", box_prec="u8", order="bfs"),
    "bvh8_soa_f16": dict(width=8, box_layout="soa", box_prec="f16"),
    "bvh8_aos_u8": dict(width=8, box_layout="aos", box_prec="u8"),
}
# Traversal parameters the batched launch honours: child order and fetch
# mode (warp batches, or warp refill once 8 lanes are idle).
CANDIDATE_PARAMS = {"ordered": {}, "slot_order": {"ordered_children": 2},
                    "nearest_first": {"ordered_children": 3},
                    "ordered_refill8": {"rays_per_fetch": 8},
                    "slot_order_refill8": {"ordered_children": 2, "rays_per_fetch": 8},
                    "nearest_first_refill8": {"ordered_children": 3, "rays_per_fetch": 8}}


@dataclass
class Choice:
    name: str
    desc: object
    params: dict
    bvh: object
    times_ms: dict = field(default_factory=dict)


class Autotuner:
    """Candidates are timed through the batched kernel itself (a batch of the
    one scene and its ray sample), so the choice is what the batched launch
    will run; `plain=True` times plain launches instead."""

    def __init__(self, prim_refs=("direct",), params=None, sample: int = 8192, reps: int = 3,
                 layouts=None, plain: bool = False):
        self.descs = {}
        for name, kw in (layouts or CANDIDATE_LAYOUTS).items():
            for pr in prim_refs:
                self.descs[f"{name}_{pr}"] = scion.layout(prim_ref=pr, **kw)
        self.params = params if params is not None else CANDIDATE_PARAMS
        self.sample = sample
        self.reps = reps
        self.plain = plain
        self.cache = {}

    def _time(self, bvh, rays, params, out):
        import torch
        if self.plain:
            def run():
                scion.scion_trace_closest(bvh, rays, out, params=params or None)
        else:
            batch = scion.Batch([bvh], [rays], hits=[out], params=[params or {}])
            run = batch.launch
        best = None
        for _ in range(self.reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run()
            b.record()
            b.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        return best

    def tune(self, key, verts, indices, rays) -> Choice:
        """Pick (layout, params) for one scene; returns the chosen BVH."""
        import torch
        names = list(self.descs)
        if key in self.cache:
            name, pname = self.cache[key]
            bvh = scion.scion_build(verts, self.descs[name], indices)
            return Choice(name, self.descs[name], self.params[pname], bvh)
        bvhs = scion.scion_build_many(verts, [self.descs[n] for n in names], indices)
        n = rays.shape[0]
        step = max(1, n // self.sample)
        sample = rays[::step][: self.sample].contiguous()
        out = torch.empty((sample.shape[0], 4), dtype=torch.int32, device=rays.device)
        times = {}
        for name, bvh in zip(names, bvhs):
            for pname, p in self.params.items():
                times[(name, pname)] = self._time(bvh, sample, p, out)
        best = min(times, key=times.get)
        self.cache[key] = best
        chosen = bvhs[names.index(best[0])]
        for b in bvhs:
            if b is not chosen:
                scion.scion_destroy(b)
        return Choice(best[0], self.descs[best[0]], self.params[best[1]], chosen,
                      {f"{a}/{b}": t for (a, b), t in times.items()})
