"""CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package. The product library never calls it and
shares no code with it.

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``;
the functions below marshal numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SRC = os.path.join(HERE, "oracle.c")
MISS = 0xFFFFFFFF

HIT_DTYPE = np.dtype([("t", np.float32), ("u", np.float32), ("v", np.float32), ("prim", np.uint32)])

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(SRC),
                                                 os.path.getmtime(os.path.join(HERE, "oracle.h")))):
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _bind(path):
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    U64 = ctypes.c_uint64
    I = ctypes.c_int
    L.oracle_intersect.argtypes = [P, P, P, P, P]
    L.oracle_intersect.restype = I
    L.oracle_closest_brute.argtypes = [P, U64, P, U64, P, I]
    L.oracle_any_brute.argtypes = [P, U64, P, U64, P, I]
    L.oracle_bvh_build.argtypes = [P, U64, I, I]
    L.oracle_bvh_build.restype = P
    L.oracle_bvh_closest.argtypes = [P, P, U64, P, I]
    L.oracle_bvh_any.argtypes = [P, P, U64, P, I]
    L.oracle_bvh_stats.argtypes = [P, P, P, P]
    L.oracle_bvh_free.argtypes = [P]
    L.oracle_grad.argtypes = [P, P, U64, P, P, P, U64, P, P]
    L.oracle_grad_fd.argtypes = [P, P, U64, P, P, P, U64, ctypes.c_double, P, P]
    L.oracle_plane_tuv.argtypes = [P, P, P, P, P, P]
    L.oracle_plane_tuv.restype = I
    L.oracle_max_threads.restype = I
    L.oracle_cpq_brute.argtypes = [P, U64, P, U64, P, I]
    L.oracle_closest_point.argtypes = [P, P, P, P, P]
    L.oracle_closest_point.restype = I
    return L


def use_library(path):
    """Swap in another build of oracle.c (the mutation tests use this to check
    that planted mistakes fail the pins). Returns the previous library."""
    global _lib
    prev = _lib
    _lib = _bind(path) if path else None
    return prev


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def intersect(ray, tri):
    """One ray (8 floats) against one triangle (9 floats): (t, u, v) or None."""
    r = _f32(ray).reshape(8)
    p = _f32(tri).reshape(9)
    out = np.zeros(3, np.float32)
    o = [out[i:i + 1] for i in range(3)]
    ok = lib().oracle_intersect(_ptr(r), _ptr(p), _ptr(o[0]), _ptr(o[1]), _ptr(o[2]))
    return (float(out[0]), float(out[1]), float(out[2])) if ok else None


def closest_brute(tris, rays, threads: int = 0) -> np.ndarray:
    tris = _f32(tris).reshape(-1, 9)
    rays = _f32(rays).reshape(-1, 8)
    hits = np.zeros(rays.shape[0], HIT_DTYPE)
    lib().oracle_closest_brute(_ptr(tris), tris.shape[0], _ptr(rays), rays.shape[0], _ptr(hits), threads)
    return hits


def any_brute(tris, rays, threads: int = 0) -> np.ndarray:
    tris = _f32(tris).reshape(-1, 9)
    rays = _f32(rays).reshape(-1, 8)
    occ = np.zeros(rays.shape[0], np.uint32)
    lib().oracle_any_brute(_ptr(tris), tris.shape[0], _ptr(rays), rays.shape[0], _ptr(occ), threads)
    return occ


class BVH2:
    """The oracle's own binned-SAH BVH2 with the paper's recursive traversal."""

    def __init__(self, tris, bins: int = 32, leaf_max: int = 4):
        self._tris = _f32(tris).reshape(-1, 9)
        self._h = lib().oracle_bvh_build(_ptr(self._tris), self._tris.shape[0], bins, leaf_max)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_bvh_free(self._h)
            self._h = None

    def stats(self):
        n = np.zeros(1, np.uint64)
        d = np.zeros(1, np.uint32)
        s = np.zeros(1, np.uint64)
        lib().oracle_bvh_stats(self._h, _ptr(n), _ptr(d), _ptr(s))
        return {"n_nodes": int(n[0]), "depth": int(d[0]), "leaf_tris": int(s[0])}

    def closest(self, rays, threads: int = 0) -> np.ndarray:
        rays = _f32(rays).reshape(-1, 8)
        hits = np.zeros(rays.shape[0], HIT_DTYPE)
        lib().oracle_bvh_closest(self._h, _ptr(rays), rays.shape[0], _ptr(hits), threads)
        return hits

    def any(self, rays, threads: int = 0) -> np.ndarray:
        rays = _f32(rays).reshape(-1, 8)
        occ = np.zeros(rays.shape[0], np.uint32)
        lib().oracle_bvh_any(self._h, _ptr(rays), rays.shape[0], _ptr(occ), threads)
        return occ


def _grad_common(fn, tris, tri_verts, n_verts, rays, hits, grad_tuv, *extra):
    tris = _f32(tris).reshape(-1, 9)
    rays = _f32(rays).reshape(-1, 8)
    hits = np.ascontiguousarray(hits, HIT_DTYPE)
    g = _f32(grad_tuv).reshape(-1, 3)
    tv = None if tri_verts is None else np.ascontiguousarray(tri_verts, np.uint32).reshape(-1, 3)
    hit = hits["prim"] != MISS
    if np.any(hits["prim"][hit] >= tris.shape[0]):
        raise ValueError("hit prim out of range")
    gv = np.zeros((n_verts, 3), np.float64)
    gr = np.zeros((rays.shape[0], 6), np.float64)
    fn(_ptr(tris), _ptr(tv), n_verts, _ptr(rays), _ptr(hits), _ptr(g), rays.shape[0], *extra,
       _ptr(gv), _ptr(gr))
    return gv, gr


def grad(tris, tri_verts, n_verts, rays, hits, grad_tuv):
    """FP64 analytic gradient: (dL/dverts [n_verts,3], dL/drays [n,6])."""
    return _grad_common(lib().oracle_grad, tris, tri_verts, n_verts, rays, hits, grad_tuv)


def grad_fd(tris, tri_verts, n_verts, rays, hits, grad_tuv, h: float = 1e-3):
    """Central differences of the FP64 plane intersection (triangle fixed)."""
    return _grad_common(lib().oracle_grad_fd, tris, tri_verts, n_verts, rays, hits, grad_tuv,
                        ctypes.c_double(h))


def plane_tuv(o, d, p0, p1, p2):
    a = [np.ascontiguousarray(x, np.float64).reshape(3) for x in (o, d, p0, p1, p2)]
    out = np.zeros(3, np.float64)
    ok = lib().oracle_plane_tuv(*[_ptr(x) for x in a], _ptr(out))
    return tuple(out) if ok else None


def closest_point(pt, tri):
    """One point (3 floats) against one triangle (9 floats): (d2, u, v), or
    None for a non-finite triangle."""
    p = _f32(pt).reshape(3)
    t = _f32(tri).reshape(9)
    out = np.zeros(3, np.float32)
    o = [out[i:i + 1] for i in range(3)]
    ok = lib().oracle_closest_point(_ptr(p), _ptr(t), _ptr(o[0]), _ptr(o[1]), _ptr(o[2]))
    return (float(out[0]), float(out[1]), float(out[2])) if ok else None


def cpq_brute(tris, points, threads: int = 0) -> np.ndarray:
    """Closest point query by brute force. points: float [n][4] (x, y, z,
    r2max). Returns records (t = d2, u, v, prim) in the hit dtype."""
    tris = _f32(tris).reshape(-1, 9)
    pts = _f32(points).reshape(-1, 4)
    out = np.zeros(pts.shape[0], HIT_DTYPE)
    lib().oracle_cpq_brute(_ptr(tris), tris.shape[0], _ptr(pts), pts.shape[0], _ptr(out), threads)
    return out
