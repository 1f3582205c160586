"""Refit: the same tree with new vertex positions. After scion_refit every
layout family must trace the moved scene bit-identically to the CPU oracle
(boxes recomputed bottom-up and re-encoded in place, rounded outward), for
small and large motions, repeated refits, GPU-built trees, and vertices that
become non-finite."""
import ctypes

import numpy as np
import pytest

from layout_cases import all_layouts
from paper_2511_15028_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# one of each node codec x layout form x reference kind, plus orders
CASES = [kw for kw in all_layouts()
         if kw["order"] == "dfs" or (kw["box_prec"] == "u8" and kw["width"] == 8)]


@pytest.fixture(scope="module")
def sc_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15028_gb300 import build as b
    b.build()
    from paper_2511_15028_gb300 import scion
    scion.lib()
    return scion


def moved(verts, amp, scale=1.0, shift=(0.0, 0.0, 0.0)):
    v = verts.astype(np.float64)
    w = v.copy()
    w[:, 2] += amp * np.sin(5.0 * v[:, 0]) * np.cos(3.0 * v[:, 1])
    w[:, 0] += 0.5 * amp * np.cos(4.0 * v[:, 2])
    return (w * scale + np.asarray(shift)).astype(np.float32)


def rays_for(verts, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = verts.min(0) - 0.2, verts.max(0) + 0.2
    return scenes.random_rays(rng, n, lo, hi)


def check(scion, oracle, bvh, verts, indices, rays, what):
    tris = verts[indices].reshape(-1, 9) if indices is not None else verts.reshape(-1, 9)
    exp = oracle.closest_brute(tris, rays)
    occ = oracle.any_brute(tris, rays)
    d = torch.from_numpy(rays).cuda()
    got = scion.scion_trace_closest(bvh, d).cpu().numpy().view(np.uint32).reshape(-1, 4)
    e = np.ascontiguousarray(exp).view(np.uint32).reshape(-1, 4)
    bad = np.where(np.any(got != e, axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} of {len(e)} rays differ, first {bad[:5]}"
    assert np.array_equal(scion.scion_trace_any(bvh, d).cpu().numpy().astype(np.uint32), occ), what
    assert scion.scion_get_status(bvh) == 0, what


@pytest.mark.parametrize("kw", CASES, ids=lambda kw: "-".join(str(v) for v in kw.values()))
def test_refit_every_layout(sc_mod, oracle_mod, kw):
    sc = scenes.config1_scene()
    bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(**kw), sc.indices)
    v1 = moved(sc.verts, 0.15)
    sc_mod.scion_refit(bvh, torch.from_numpy(v1).cuda())
    check(sc_mod, oracle_mod, bvh, v1, sc.indices, scenes.config1_rays(), f"{kw} small motion")
    # a large motion moves the world grid (q16 / eq10) and every u8 frame
    v2 = moved(sc.verts, 0.6, scale=3.0, shift=(10.0, -4.0, 2.5))
    sc_mod.scion_refit(bvh, torch.from_numpy(v2).cuda())
    check(sc_mod, oracle_mod, bvh, v2, sc.indices, rays_for(v2, 8192, 1), f"{kw} large motion")


def test_refit_back_and_soup_and_gpu_built(sc_mod, oracle_mod):
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    for kw in (dict(width=8, box_prec="u8", prim_ref="direct"), dict(box_prec="q16", box_layout="soa")):
        bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(**kw), sc.indices)
        before = sc_mod.scion_trace_closest(bvh, torch.from_numpy(rays).cuda()).cpu()
        sc_mod.scion_refit(bvh, torch.from_numpy(moved(sc.verts, 0.3)).cuda())
        sc_mod.scion_refit(bvh, torch.from_numpy(sc.verts).cuda())
        after = sc_mod.scion_trace_closest(bvh, torch.from_numpy(rays).cuda()).cpu()
        assert torch.equal(before, after), kw  # same boxes as the build, same hits
    # a soup built on the GPU, refit twice
    rng = scenes.rng_for(9)
    soup = scenes.random_soup(rng, 20000, mu=np.log(0.02))
    r = scenes.random_rays(rng, 8192, (0, 0, 0), (1, 1, 1))
    bvh = sc_mod.scion_build_gpu(torch.from_numpy(soup).cuda(), sc_mod.layout(width=4, box_layout="soa"))
    for k in range(2):
        v = moved(soup, 0.05 * (k + 1))
        sc_mod.scion_refit(bvh, torch.from_numpy(v).cuda())
        check(sc_mod, oracle_mod, bvh, v, None, r, f"gpu-built soup refit {k}")


def test_refit_nonfinite_and_arguments(sc_mod, oracle_mod):
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    for kw in (dict(), dict(width=8, box_prec="f16", box_layout="soa"), dict(box_prec="eq10")):
        bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(**kw), sc.indices)
        v = sc.verts.copy()
        v[100] = np.nan  # the triangles on this vertex are never hit from now on
        v[2000, 2] = np.inf
        sc_mod.scion_refit(bvh, torch.from_numpy(v).cuda())
        check(sc_mod, oracle_mod, bvh, v, sc.indices, rays, f"{kw} non-finite")
    L = sc_mod.lib()
    d = torch.from_numpy(sc.verts).cuda()
    assert L.scion_refit(bvh.handle, ctypes.c_void_p(d.data_ptr()), d.shape[0] - 1, None) == 1
    assert L.scion_refit(bvh.handle, sc.verts.ctypes.data_as(ctypes.c_void_p), sc.verts.shape[0], None) == 1
