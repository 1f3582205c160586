"""Python binding of the scion C ABI (include/scion.h, include/scion_debug.h).

Argument marshalling only: every step of build, packing and traversal runs in
the native library ``_build/libscion.so`` (host C++ builder, CUDA kernels for
sm_103a). PyTorch provides device memory and streams. There is no fallback:
if the library is missing or fails to load, every call raises.

The functions carry the C names: ``scion_build``, ``scion_bvh_info``,
``scion_trace_closest``, ``scion_trace_any``, ``scion_get_status``,
``scion_destroy``, plus the host-only ``scion_debug_*`` introspection calls.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libscion.so")

SCION_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_LAYOUT", 3: "OOM", 4: "CUDA",
                5: "STACK_OVERFLOW", 6: "ITER_LIMIT", 7: "BAD_INPUT"}
PRIM_MISS = 0xFFFFFFFF
PRIM_ERROR = 0xFFFFFFFE


class ScionError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} ({last_error()})")


class LayoutDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "width", "box_layout", "box_prec", "child_ref", "prim_ref", "order", "leaf_max",
        "sah_bins", "treelet_bytes", "align")]


class TraceParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "threads_per_block", "ctas_per_sm", "reg_stack", "smem_stack", "ordered_children",
        "rays_per_fetch", "max_steps", "raster_width")]


class DebugInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint32), ("node_stride", ctypes.c_uint32),
                ("n_leaf_entries", ctypes.c_uint32), ("root_ref", ctypes.c_uint32),
                ("depth", ctypes.c_uint32), ("stack_need", ctypes.c_uint32),
                ("own_box", ctypes.c_uint32), ("node2_bytes", ctypes.c_uint32),
                ("node_bytes", ctypes.c_uint64), ("prim_bytes", ctypes.c_uint64),
                ("vert_bytes", ctypes.c_uint64), ("build_ms", ctypes.c_double)]


PREC = {"f32": 0, "f16": 1, "u8": 2, "q16": 3, "eq10": 4, "u16": 5, "slab": 6}
ORDER = {"dfs": 0, "bfs": 1, "treelet": 2}


def layout(width=2, box_layout="aos", box_prec="f32", child_ref="direct", prim_ref="indirect",
           order="dfs", leaf_max=4, sah_bins=16, treelet_bytes=1024, align=0) -> LayoutDesc:
    """A layout descriptor from readable names."""
    return LayoutDesc(width, 0 if box_layout == "aos" else 1, PREC[box_prec],
                      0 if child_ref == "direct" else 1, 0 if prim_ref == "direct" else 1,
                      ORDER[order], leaf_max, sah_bins, treelet_bytes, align)


# The four node layouts swept on the coherent/incoherent workloads, each with
# direct and indirect triangle storage.
SWEEP = {
    "bvh2_aos_f32": dict(width=2, box_layout="aos", box_prec="f32"),
    "bvh4_soa_f32": dict(width=4, box_layout="soa", box_prec="f32"),
    "bvh8_soa_f16": dict(width=8, box_layout="soa", box_prec="f16"),
    "bvh8_aos_u8": dict(width=8, box_layout="aos", box_prec="u8"),
}


# Further layouts: the world-grid quantised bvh2 layouts of Table 1 (Section
# 9.2.5, App. D.1, D.3: sg-pbrt-q16, sg-pbrt-q16-soaos, sg-eq, sg-eq-align16),
# the 16-bit parent-relative 8-wide node (bvh8-q16) and the shared-slab bvh2
# node with tree-carried bounds (Section 8.3).
SWEEP_EXTENDED = {
    "bvh2_aos_q16": dict(width=2, box_layout="aos", box_prec="q16"),
    "bvh2_soa_q16": dict(width=2, box_layout="soa", box_prec="q16"),
    "bvh2_aos_eq10": dict(width=2, box_layout="aos", box_prec="eq10"),
    "bvh2_aos_eq10_a16": dict(width=2, box_layout="aos", box_prec="eq10", align=16),
    "bvh8_aos_u16": dict(width=8, box_layout="aos", box_prec="u16"),
    "bvh8_soa_u8": dict(width=8, box_layout="soa", box_prec="u8"),
    "bvh2_slab": dict(width=2, box_layout="aos", box_prec="slab"),
}


# Breadth-first node order for the wide layouts (the order axis: the levels
# every ray visits sit together at the front of the node buffer instead of
# being spread through it by depth-first subtrees).
SWEEP_ORDER = {
    "bvh4_soa_f32_bfs": dict(width=4, box_layout="soa", box_prec="f32", order="bfs"),
    # 4-wide nodes of 64 bytes (two 256-bit loads instead of four)
    "bvh4_soa_f16_bfs": dict(width=4, box_layout="soa", box_prec="f16", order="bfs"),
    "bvh4_soa_u8_bfs": dict(width=4, box_layout="soa", box_prec="u8", order="bfs"),
    "bvh8_soa_f16_bfs": dict(width=8, box_layout="soa", box_prec="f16", order="bfs"),
    "bvh8_aos_u8_bfs": dict(width=8, box_layout="aos", box_prec="u8", order="bfs"),
}


def sweep_layouts(extended: bool = False, orders: bool = False):
    """Named descriptors of the swept layouts, each with direct and indirect
    triangle storage (plus the further Table 1 layouts and the breadth-first
    orders if asked)."""
    out = {}
    sweep = dict(SWEEP, **SWEEP_EXTENDED) if extended else dict(SWEEP)
    if orders:
        sweep.update(SWEEP_ORDER)
    for name, kw in sweep.items():
        for pr in ("direct", "indirect"):
            out[f"{name}_{pr}"] = layout(prim_ref=pr, **kw)
    return out


_lib = None


def lib():
    """Load the native library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"native library missing: {LIB_PATH}; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.scion_build.argtypes = [P, U64, P, U64, ctypes.POINTER(LayoutDesc), P, ctypes.POINTER(P)]
        L.scion_build_gpu.argtypes = [P, U64, P, U64, ctypes.POINTER(LayoutDesc), P, ctypes.POINTER(P)]
        L.scion_bvh_build_times.argtypes = [P, P, P]
        L.scion_refit.argtypes = [P, P, U64, P]
        L.scion_query_closest_point.argtypes = [P, P, U64, P, P, P]
        L.scion_bvh_info.argtypes = [P, P, P, P, P]
        L.scion_build_many.argtypes = [P, U64, P, U64, ctypes.POINTER(LayoutDesc), U32, P, ctypes.POINTER(P)]
        L.scion_trace_closest.argtypes = [P, P, U64, P, ctypes.POINTER(TraceParams), P]
        L.scion_trace_any.argtypes = [P, P, U64, P, ctypes.POINTER(TraceParams), P]
        L.scion_get_status.argtypes = [P, P, P]
        L.scion_trace_stats.argtypes = [P, P, U64, U32, P, ctypes.POINTER(TraceParams), P, P]
        L.scion_trace_backward.argtypes = [P, P, P, P, U64, P, P, P]
        L.scion_batch_create.argtypes = [P, P, P, P, U32, P, P, ctypes.POINTER(P)]
        L.scion_batch_launch.argtypes = [P, P]
        L.scion_batch_info.argtypes = [P, P, P]
        L.scion_batch_destroy.argtypes = [P]
        L.scion_batch_destroy.restype = None
        L.scion_trace_batched.argtypes = [P, P, P, P, U32, P, P]
        L.scion_destroy.argtypes = [P]
        L.scion_destroy.restype = None
        L.scion_status_string.argtypes = [I]
        L.scion_status_string.restype = ctypes.c_char_p
        L.scion_last_error.restype = ctypes.c_char_p
        L.scion_debug_build_host.argtypes = [P, U64, P, U64, ctypes.POINTER(LayoutDesc), ctypes.POINTER(P)]
        L.scion_debug_host_stats.argtypes = [P, ctypes.POINTER(DebugInfo)]
        L.scion_debug_host_decode.argtypes = [P, P, P, P, P, P, P]
        L.scion_debug_host_raw.argtypes = [P, P, U64, P, U64, P]
        L.scion_debug_host_destroy.argtypes = [P]
        L.scion_debug_host_destroy.restype = None
        L.scion_debug_f16_round.argtypes = [ctypes.c_float, I]
        L.scion_debug_f16_round.restype = U32
        L.scion_debug_raster_slots.argtypes = [U64, U32]
        L.scion_debug_raster_slots.restype = U64
        L.scion_debug_build_gpu_host_pack.argtypes = [P, U64, P, U64, ctypes.POINTER(LayoutDesc), P,
                                                      ctypes.POINTER(P)]
        L.scion_debug_build_gpu_host_pack.restype = I
        L.scion_debug_bvh_bytes.argtypes = [P, P, U64, P, U64, P, U64, P]
        L.scion_debug_bvh_bytes.restype = I
        L.scion_debug_read_bandwidth.argtypes = [P, U64, U32, P, P]
        L.scion_debug_read_bandwidth.restype = I
        L.scion_debug_f16_decode.argtypes = [U32]
        L.scion_debug_f16_decode.restype = ctypes.c_float
        for name in ("scion_build", "scion_build_gpu", "scion_bvh_build_times", "scion_refit",
                     "scion_query_closest_point",
                     "scion_build_many", "scion_bvh_info", "scion_trace_closest", "scion_trace_any",
                     "scion_trace_stats", "scion_trace_backward", "scion_batch_create",
                     "scion_batch_launch", "scion_batch_info", "scion_trace_batched",
                     "scion_get_status", "scion_debug_build_host", "scion_debug_host_stats",
                     "scion_debug_host_decode", "scion_debug_host_raw"):
            getattr(L, name).restype = I
        _lib = L
    return _lib


def last_error() -> str:
    try:
        return lib().scion_last_error().decode()
    except Exception:  # noqa: BLE001 - message helper only
        return ""


def _check(st: int, what: str):
    if st != SCION_OK:
        raise ScionError(st, what)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class BVH:
    """Owning handle of a device BVH (scion_bvh)."""

    def __init__(self, handle, n_tris: int, n_verts: int, desc: LayoutDesc):
        self.handle = handle
        self.n_tris = n_tris
        self.n_verts = n_verts
        self.desc = desc

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.scion_destroy(self.handle)
            self.handle = None

    def info(self):
        return scion_bvh_info(self)


def _as_np(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def scion_build(verts, desc: LayoutDesc, indices=None, stream=None) -> BVH:
    """Build a BVH from float32 vertices [n_verts, 3] (numpy or torch, host or
    device) and optional uint32 indices [n_tris, 3]."""
    import torch
    keep = []

    def ptr(x, dtype):
        if x is None:
            return None, 0
        if isinstance(x, torch.Tensor):
            t = x.contiguous()
            keep.append(t)
            return ctypes.c_void_p(t.data_ptr()), t.shape[0]
        a = _as_np(x, dtype)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p), a.shape[0]

    vp, nv = ptr(verts, np.float32)
    ip, nt = ptr(indices, np.uint32)
    if indices is None:
        nt = nv // 3
    h = ctypes.c_void_p()
    _check(lib().scion_build(vp, nv, ip, nt, ctypes.byref(desc), _stream_ptr(stream), ctypes.byref(h)),
           "scion_build")
    return BVH(h, nt, nv, desc)


def scion_build_gpu(verts, desc: LayoutDesc, indices=None, stream=None, host_pack: bool = False) -> BVH:
    """Build with the logical BVH2 constructed on the GPU (linear BVH) and
    packed into `desc` on the GPU (host_pack=True: by the host packers, the
    debug reference). verts: float32 [n_verts, 3] and indices: int32/uint32
    [n_tris, 3] (or None for a soup), CUDA tensors or numpy arrays (copied to
    the device first)."""
    import torch
    v = torch.as_tensor(verts, dtype=torch.float32).cuda().contiguous()
    ix = None
    if indices is not None:
        if isinstance(indices, torch.Tensor):
            ix = indices.to(torch.int32)  # same bits as uint32 below 2^31
        else:
            ix = torch.from_numpy(_as_np(indices, np.uint32).view(np.int32))
        ix = ix.cuda().contiguous()
    nv = v.shape[0]
    nt = nv // 3 if ix is None else ix.shape[0]
    h = ctypes.c_void_p()
    fn = lib().scion_debug_build_gpu_host_pack if host_pack else lib().scion_build_gpu
    _check(fn(ctypes.c_void_p(v.data_ptr()), nv, None if ix is None else ctypes.c_void_p(ix.data_ptr()), nt,
              ctypes.byref(desc), _stream_ptr(stream), ctypes.byref(h)), "scion_build_gpu")
    return BVH(h, nt, nv, desc)


def scion_debug_bvh_bytes(bvh: BVH):
    """(nodes, nodes2, prims) byte arrays copied from a BVH's device buffers."""
    sizes = (ctypes.c_uint64 * 3)()
    _check(lib().scion_debug_bvh_bytes(bvh.handle, None, 0, None, 0, None, 0, sizes), "scion_debug_bvh_bytes")
    bufs = [np.zeros(max(int(n), 1), np.uint8) for n in sizes]
    P = lambda x: x.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().scion_debug_bvh_bytes(bvh.handle, P(bufs[0]), bufs[0].size, P(bufs[1]), bufs[1].size,
                                       P(bufs[2]), bufs[2].size, sizes), "scion_debug_bvh_bytes")
    return tuple(b[:int(n)] for b, n in zip(bufs, sizes))


def scion_refit(bvh: BVH, verts, stream=None) -> None:
    """Refit `bvh` to new vertex positions (float32 [n_verts, 3], CUDA tensor
    or numpy array copied to the device): same triangles, same tree."""
    import torch
    v = torch.as_tensor(verts, dtype=torch.float32).cuda().contiguous()
    _check(lib().scion_refit(bvh.handle, ctypes.c_void_p(v.data_ptr()), v.shape[0], _stream_ptr(stream)),
           "scion_refit")
    bvh._refit_src = v  # keep the source alive until the enqueued copies ran


def scion_bvh_build_times(bvh: BVH) -> dict:
    """{'logical_ms', 'pack_ms'}: logical BVH2 construction (host SAH wall
    time or GPU build device time) and host packing."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().scion_bvh_build_times(bvh.handle, ctypes.byref(a), ctypes.byref(b)), "scion_bvh_build_times")
    return {"logical_ms": a.value, "pack_ms": b.value}


def scion_build_many(verts, descs, indices=None, stream=None):
    """Several layouts of one scene from a single logical build: list of BVH."""
    import torch
    keep = []

    def ptr(x, dtype):
        if x is None:
            return None, 0
        if isinstance(x, torch.Tensor):
            t = x.contiguous()
            keep.append(t)
            return ctypes.c_void_p(t.data_ptr()), t.shape[0]
        a = _as_np(x, dtype)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p), a.shape[0]

    vp, nv = ptr(verts, np.float32)
    ip, nt = ptr(indices, np.uint32)
    if indices is None:
        nt = nv // 3
    arr = (LayoutDesc * len(descs))(*descs)
    hs = (ctypes.c_void_p * len(descs))()
    _check(lib().scion_build_many(vp, nv, ip, nt, arr, len(descs), _stream_ptr(stream), hs), "scion_build_many")
    return [BVH(ctypes.c_void_p(h), nt, nv, d) for h, d in zip(hs, descs)]


def scion_bvh_info(bvh: BVH) -> dict:
    nb, pb = ctypes.c_uint64(), ctypes.c_uint64()
    d, n = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().scion_bvh_info(bvh.handle, ctypes.byref(nb), ctypes.byref(pb), ctypes.byref(d),
                                ctypes.byref(n)), "scion_bvh_info")
    return {"node_bytes": nb.value, "prim_bytes": pb.value, "depth": d.value, "n_nodes": n.value}


def _params(params):
    if params is None:
        return None
    if isinstance(params, TraceParams):
        return ctypes.byref(params)
    return ctypes.byref(TraceParams(**params))


def _ray_buffer(t, dtype):
    """Device tensors, or pinned host tensors that the kernel reads and
    writes in place."""
    if not (t.is_cuda or t.is_pinned()) or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor on the GPU or in pinned host memory, got "
                        f"{t.dtype} on {t.device}{'' if t.is_contiguous() else ' (not contiguous)'}")


def _device_buffer(t, dtype):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor on the GPU, got {t.dtype} on {t.device}")


def _like(rays, shape, dtype):
    import torch
    if rays.is_cuda:
        return torch.empty(shape, dtype=dtype, device=rays.device)
    return torch.empty(shape, dtype=dtype).pin_memory()


def scion_trace_closest(bvh: BVH, rays, hits=None, params=None, stream=None):
    """Closest hits of rays (float32 [n, 8], on the device or in pinned host
    memory); returns int32 [n, 4] beside them holding (t, u, v) as float bits
    and prim as uint32 bits."""
    import torch
    _ray_buffer(rays, torch.float32)
    n = rays.shape[0]
    if hits is None:
        hits = _like(rays, (n, 4), torch.int32)
    _ray_buffer(hits, torch.int32)
    _check(lib().scion_trace_closest(bvh.handle, ctypes.c_void_p(rays.data_ptr()), n,
                                     ctypes.c_void_p(hits.data_ptr()), _params(params),
                                     _stream_ptr(stream)), "scion_trace_closest")
    return hits


def scion_trace_any(bvh: BVH, rays, occluded=None, params=None, stream=None):
    """Any-hit flags (int32 [n]: 1 occluded, 0 clear) of rays on the device or
    in pinned host memory."""
    import torch
    _ray_buffer(rays, torch.float32)
    n = rays.shape[0]
    if occluded is None:
        occluded = _like(rays, (n,), torch.int32)
    _ray_buffer(occluded, torch.int32)
    _check(lib().scion_trace_any(bvh.handle, ctypes.c_void_p(rays.data_ptr()), n,
                                 ctypes.c_void_p(occluded.data_ptr()), _params(params),
                                 _stream_ptr(stream)), "scion_trace_any")
    return occluded


def scion_query_closest_point(bvh: BVH, points, out=None, params=None, stream=None):
    """Closest points of query points (float32 [n, 4]: x, y, z, r2max; on
    the device or in pinned host memory); returns int32 [n, 4] beside them
    holding (d2, u, v) as float bits and prim as uint32 bits."""
    import torch
    _ray_buffer(points, torch.float32)
    n = points.shape[0]
    if out is None:
        out = _like(points, (n, 4), torch.int32)
    _ray_buffer(out, torch.int32)
    _check(lib().scion_query_closest_point(bvh.handle, ctypes.c_void_p(points.data_ptr()), n,
                                           ctypes.c_void_p(out.data_ptr()), _params(params),
                                           _stream_ptr(stream)), "scion_query_closest_point")
    return out


def scion_trace_stats(bvh: BVH, rays, query: int = 0, params=None, stream=None):
    """Counting trace: (results, counters) with counters = int64 tensor
    [nodes fetched, leaves visited, triangles tested, rays]."""
    import torch
    _device_buffer(rays, torch.float32)
    n = rays.shape[0]
    out = (torch.empty((n,), dtype=torch.int32, device=rays.device) if query == 1
           else torch.empty((n, 4), dtype=torch.int32, device=rays.device))
    cnt = torch.zeros(4, dtype=torch.int64, device=rays.device)
    _check(lib().scion_trace_stats(bvh.handle, ctypes.c_void_p(rays.data_ptr()), n, query,
                                   ctypes.c_void_p(out.data_ptr()), _params(params), _stream_ptr(stream),
                                   ctypes.c_void_p(cnt.data_ptr())), "scion_trace_stats")
    return out, cnt


def scion_trace_backward(bvh: BVH, rays, hits, grad_tuv, grad_verts=None, grad_rays=None,
                         want_ray_grads: bool = True, stream=None):
    """Backward pass: returns (grad_verts float32 [n_verts, 3] (accumulated
    into if given), grad_rays float32 [n, 8] or None)."""
    import torch
    n = rays.shape[0]
    dev = rays.device
    g = grad_tuv.contiguous().float()
    if grad_verts is None:
        grad_verts = torch.zeros((bvh.n_verts, 3), dtype=torch.float32, device=dev)
    if grad_rays is None and want_ray_grads:
        grad_rays = torch.empty((n, 8), dtype=torch.float32, device=dev)
    _check(lib().scion_trace_backward(bvh.handle, ctypes.c_void_p(rays.data_ptr()),
                                      ctypes.c_void_p(hits.data_ptr()), ctypes.c_void_p(g.data_ptr()), n,
                                      ctypes.c_void_p(grad_verts.data_ptr()),
                                      None if grad_rays is None else ctypes.c_void_p(grad_rays.data_ptr()),
                                      _stream_ptr(stream)), "scion_trace_backward")
    return grad_verts, grad_rays


def _trace_fn():
    import torch

    class TraceFn(torch.autograd.Function):
        """Differentiable closest hit: (verts, rays) -> (t, u, v, prim).

        The forward traces with the BVH built from `verts` (the caller keeps the
        two consistent); the backward keeps every ray's hit triangle fixed and
        returns dL/dverts and dL/drays (the ray's tmin/tmax get zero)."""

        @staticmethod
        def forward(ctx, verts, rays, bvh):
            hits = scion_trace_closest(bvh, rays.detach().contiguous())
            ctx.save_for_backward(rays, hits)
            ctx.bvh = bvh
            f = hits.view(torch.float32)
            prim = hits[:, 3]
            ctx.mark_non_differentiable(prim)
            return f[:, 0].clone(), f[:, 1].clone(), f[:, 2].clone(), prim.clone()

        @staticmethod
        def backward(ctx, gt, gu, gv, _gp):
            rays, hits = ctx.saved_tensors
            n = rays.shape[0]
            z = lambda x: x if x is not None else torch.zeros(n, device=rays.device)  # noqa: E731
            g = torch.stack([z(gt), z(gu), z(gv)], -1).contiguous()
            gverts, grays = scion_trace_backward(ctx.bvh, rays.detach().contiguous(), hits, g,
                                                 want_ray_grads=ctx.needs_input_grad[1])
            return (gverts if ctx.needs_input_grad[0] else None,
                    grays if ctx.needs_input_grad[1] else None, None)

    return TraceFn


_TRACE_FN = None


def trace_fn():
    """The torch.autograd.Function class for differentiable closest hits."""
    global _TRACE_FN
    if _TRACE_FN is None:
        _TRACE_FN = _trace_fn()
    return _TRACE_FN


class Batch:
    """Many scenes in one launch (scion_batch_*). The rays and hit tensors
    must stay alive and in place while the batch exists; launch() allocates
    nothing and may be captured in a CUDA graph."""

    def __init__(self, bvhs, rays, hits=None, params=None, stream=None):
        import torch
        self.bvhs = list(bvhs)
        self.rays = [r.contiguous() for r in rays]
        self.hits = hits if hits is not None else [
            torch.empty((r.shape[0], 4), dtype=torch.int32, device=r.device) for r in self.rays]
        m = len(self.bvhs)
        hb = (ctypes.c_void_p * m)(*[b.handle.value if isinstance(b.handle, ctypes.c_void_p) else b.handle
                                     for b in self.bvhs])
        rp = (ctypes.c_void_p * m)(*[r.data_ptr() for r in self.rays])
        n = (ctypes.c_uint64 * m)(*[r.shape[0] for r in self.rays])
        hp = (ctypes.c_void_p * m)(*[h.data_ptr() for h in self.hits])
        pp = None
        if params is not None:
            pp = (TraceParams * m)(*[p if isinstance(p, TraceParams) else TraceParams(**(p or {}))
                                     for p in params])
        self._keep = (hb, rp, n, hp, pp)
        self.handle = ctypes.c_void_p()
        _check(lib().scion_batch_create(hb, rp, n, hp, m, pp, _stream_ptr(stream), ctypes.byref(self.handle)),
               "scion_batch_create")

    def launch(self, stream=None):
        _check(lib().scion_batch_launch(self.handle, _stream_ptr(stream)), "scion_batch_launch")
        return self.hits

    def info(self):
        a, b = ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().scion_batch_info(self.handle, ctypes.byref(a), ctypes.byref(b)), "scion_batch_info")
        return {"batched_scenes": a.value, "plain_scenes": b.value}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.scion_batch_destroy(self.handle)
            self.handle = None


def scion_trace_batched(bvhs, rays, hits=None, params=None, stream=None):
    """One-shot batched closest hit over many scenes; returns the hit tensors."""
    b = Batch(bvhs, rays, hits, params, stream)
    b.launch(stream)
    import torch
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return b.hits


class HostTracer:
    """Traces rays that live in pinned host memory and returns the results
    to pinned host memory, overlapping transfers with traversal: each ray set
    is cut into chunks, and chunk i's host-to-device copy, trace and
    device-to-host copy run on stream i mod n_streams, so the copies of one
    chunk overlap the traversal of the others. Device staging buffers are
    allocated once (on first use) and reused."""

    def __init__(self, n_streams: int = 3, chunk_rays: int = 1 << 20, first_chunk_rays: int = 0,
                 zero_copy: bool = False):
        """first_chunk_rays: size of the first chunk (0: chunk_rays); the
        following chunks of the first phase double up to chunk_rays, so tracing
        starts after a short copy while later chunks are large. (The copies of
        later phases are issued early and overlap the earlier traces.)"""
        import torch
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.join = torch.cuda.Stream()
        self.chunk = chunk_rays
        self.first = first_chunk_rays or chunk_rays
        # zero_copy: no staging copies; each job is one launch that reads its
        # rays from and writes its results to the pinned host buffers directly
        self.zero_copy = zero_copy
        self._rays = [None] * n_streams
        self._outs = [None] * n_streams

    def _buf(self, i, n_rows, width, dtype, which):
        import torch
        cache = self._rays if which == "rays" else self._outs
        b = cache[i]
        if b is None or b.shape[0] < n_rows or b.shape[1:] != width or b.dtype != dtype:
            shape = (max(n_rows, self.chunk),) + width
            b = torch.empty(shape, dtype=dtype, device="cuda")
            cache[i] = b
        return b[:n_rows]

    def trace(self, jobs, phases=None):
        """jobs: list of (bvh, host_rays [n, 8] float32 pinned, host_out
        pinned (int32 [n, 4] for closest, int32 [n] for any), query
        ('closest' | 'any'), params or None). phases: optional list of lists
        of job indices; the traces of a phase start only after every trace of
        the previous phase has finished (e.g. [[0], [1, 2]]: bounce and shadow
        rays that come from the primary hits), while copies are not held
        back. Default: one phase with every job. Issues everything and makes
        the current stream wait for it: the host outputs are complete once
        the current stream reaches this point (e.g. after an event on it)."""
        import torch
        cur = torch.cuda.current_stream()
        for s in self.streams:
            s.wait_stream(cur)
        if phases is None:
            phases = [list(range(len(jobs)))]
        if self.zero_copy:
            self._trace_in_place(jobs, phases, cur)
            return
        k = 0
        prev_done = None
        for pi, ph in enumerate(phases):
            traced = []
            size = self.first if pi == 0 else self.chunk  # later phases' copies run ahead
            for j in ph:
                bvh, h_rays, h_out, query, params = jobs[j]
                n = h_rays.shape[0]
                b = 0
                while b < n:
                    e = min(n, b + size)
                    size = min(self.chunk, 2 * size)
                    i = k % len(self.streams)
                    s = self.streams[i]
                    with torch.cuda.stream(s):
                        d_r = self._buf(i, e - b, (8,), torch.float32, "rays")
                        d_r.copy_(h_rays[b:e], non_blocking=True)
                        if prev_done is not None:
                            s.wait_event(prev_done)
                        if query == "closest":
                            d_o = self._buf(i, e - b, (4,), torch.int32, "outs")
                            scion_trace_closest(bvh, d_r, d_o, params=params, stream=s)
                        else:
                            d_o = self._any_buf(i, e - b)
                            scion_trace_any(bvh, d_r, d_o, params=params, stream=s)
                        if pi + 1 < len(phases):
                            ev = torch.cuda.Event()
                            ev.record(s)
                            traced.append(ev)
                        h_out[b:e].copy_(d_o, non_blocking=True)
                    k += 1
                    b = e
            if traced:
                for ev in traced:
                    self.join.wait_event(ev)
                prev_done = torch.cuda.Event()
                prev_done.record(self.join)
        for s in self.streams:
            cur.wait_stream(s)

    def _trace_in_place(self, jobs, phases, cur):
        import torch
        k = 0
        prev_done = None
        for pi, ph in enumerate(phases):
            traced = []
            for j in ph:
                bvh, h_rays, h_out, query, params = jobs[j]
                s = self.streams[k % len(self.streams)]
                k += 1
                with torch.cuda.stream(s):
                    if prev_done is not None:
                        s.wait_event(prev_done)
                    if query == "closest":
                        scion_trace_closest(bvh, h_rays, h_out, params=params, stream=s)
                    else:
                        scion_trace_any(bvh, h_rays, h_out, params=params, stream=s)
                    if pi + 1 < len(phases):
                        ev = torch.cuda.Event()
                        ev.record(s)
                        traced.append(ev)
            if traced:
                for ev in traced:
                    self.join.wait_event(ev)
                prev_done = torch.cuda.Event()
                prev_done.record(self.join)
        for s in self.streams:
            cur.wait_stream(s)

    def _any_buf(self, i, n):
        import torch
        if not hasattr(self, "_anys"):
            self._anys = [None] * len(self.streams)
        b = self._anys[i]
        if b is None or b.shape[0] < n:
            b = torch.empty((max(n, self.chunk),), dtype=torch.int32, device="cuda")
            self._anys[i] = b
        return b[:n]


def scion_get_status(bvh: BVH, stream=None) -> int:
    st = ctypes.c_int()
    _check(lib().scion_get_status(bvh.handle, _stream_ptr(stream), ctypes.byref(st)), "scion_get_status")
    return st.value


def scion_destroy(bvh: BVH):
    if bvh.handle:
        lib().scion_destroy(bvh.handle)
        bvh.handle = None


def split_hits(hits_i32) -> np.ndarray:
    """Host structured array (t, u, v float32; prim uint32) from trace output."""
    h = hits_i32.cpu().numpy() if hasattr(hits_i32, "cpu") else np.asarray(hits_i32)
    out = np.empty(h.shape[0], dtype=[("t", np.float32), ("u", np.float32), ("v", np.float32),
                                      ("prim", np.uint32)])
    out.view(np.int32).reshape(-1, 4)[:] = h
    return out


# ------------------------------------------------------------- host debug ABI
@dataclass
class HostDecode:
    info: dict
    kind: np.ndarray
    a: np.ndarray
    c: np.ndarray
    boxes: np.ndarray
    own_boxes: np.ndarray
    leaf_ids: np.ndarray
    nodes: np.ndarray = None    # raw node array bytes
    nodes2: np.ndarray = None   # raw second node array bytes (own-box SoA)
    frame: np.ndarray = None    # world grid of the quantised own-box codecs


def scion_debug_build_host(verts, desc: LayoutDesc, indices=None) -> HostDecode:
    """Pack on the host only and decode every node (no GPU involved)."""
    v = _as_np(verts, np.float32)
    ix = None if indices is None else _as_np(indices, np.uint32)
    nt = v.shape[0] // 3 if ix is None else ix.shape[0]
    h = ctypes.c_void_p()
    _check(lib().scion_debug_build_host(v.ctypes.data_as(ctypes.c_void_p), v.shape[0],
                                        None if ix is None else ix.ctypes.data_as(ctypes.c_void_p),
                                        nt, ctypes.byref(desc), ctypes.byref(h)), "scion_debug_build_host")
    try:
        inf = DebugInfo()
        _check(lib().scion_debug_host_stats(h, ctypes.byref(inf)), "scion_debug_host_stats")
        info = {k: getattr(inf, k) for k, _ in DebugInfo._fields_}
        nn = inf.n_nodes
        kind = np.zeros(nn * 8, np.uint32)
        a = np.zeros(nn * 8, np.uint32)
        c = np.zeros(nn * 8, np.uint32)
        boxes = np.zeros(nn * 8 * 6, np.float32)
        own = np.zeros(nn * 6, np.float32)
        ids = np.zeros(max(inf.n_leaf_entries, 1), np.uint32)
        P = lambda x: x.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(lib().scion_debug_host_decode(h, P(kind), P(a), P(c), P(boxes), P(own), P(ids)),
               "scion_debug_host_decode")
        n1 = inf.node_bytes - inf.node2_bytes
        raw1 = np.zeros(max(n1, 1), np.uint8)
        raw2 = np.zeros(max(inf.node2_bytes, 1), np.uint8)
        frame = np.zeros(9, np.float32)
        _check(lib().scion_debug_host_raw(h, P(raw1), n1, P(raw2), inf.node2_bytes, P(frame)),
               "scion_debug_host_raw")
    finally:
        lib().scion_debug_host_destroy(h)
    return HostDecode(info, kind.reshape(nn, 8), a.reshape(nn, 8), c.reshape(nn, 8),
                      boxes.reshape(nn, 8, 6), own.reshape(nn, 6), ids[:inf.n_leaf_entries],
                      raw1[:n1], raw2[:inf.node2_bytes], frame)


def scion_debug_read_bandwidth(buf, reps: int, sink, stream=None) -> None:
    """Launch the L2 read probe over the device tensor `buf` (its whole
    storage, a multiple of 16 bytes) `reps` times; `sink` is a device int32
    tensor the kernel may write. The caller times the launch."""
    import torch
    if not buf.is_cuda or not buf.is_contiguous() or not sink.is_cuda:
        raise TypeError("scion_debug_read_bandwidth takes contiguous device tensors")
    nbytes = buf.numel() * buf.element_size()
    _check(lib().scion_debug_read_bandwidth(ctypes.c_void_p(buf.data_ptr()), nbytes, int(reps),
                                            ctypes.c_void_p(sink.data_ptr()), _stream_ptr(stream)),
           "scion_debug_read_bandwidth")
    del torch


def scion_debug_f16_round(x: float, direction: int) -> int:
    return int(lib().scion_debug_f16_round(float(x), int(direction)))


def scion_debug_f16_decode(h: int) -> float:
    return float(lib().scion_debug_f16_decode(int(h)))
