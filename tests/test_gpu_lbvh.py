"""GPU construction of the logical BVH2 (linear BVH: Morton order, radix tree,
bottom-up boxes) packed by the same packers: traversal results must be
bit-identical to the CPU oracle on every layout family, the tree must hold
every finite triangle exactly once (2n - 1 nodes for the own-box BVH2), and
degenerate inputs (Morton ties, non-finite vertices, empty and one-triangle
scenes) must build."""
import ctypes
import math

import numpy as np
import pytest

from paper_2511_15028_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAYOUTS = [dict(), dict(width=4, box_layout="soa", prim_ref="direct"), dict(width=8, box_prec="u8"),
           dict(width=8, box_prec="f16", box_layout="soa", child_ref="indirect", order="bfs"),
           dict(box_prec="q16"), dict(box_prec="eq10", align=16), dict(width=2, box_prec="u8")]


@pytest.fixture(scope="module")
def sc_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15028_gb300 import build as b
    b.build()
    from paper_2511_15028_gb300 import scion
    scion.lib()
    return scion


def hits(scion, bvh, rays, params=None):
    out = scion.scion_trace_closest(bvh, torch.from_numpy(rays).cuda(), params=params)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).reshape(-1, 4)


def occluded(scion, bvh, rays, params=None):
    out = scion.scion_trace_any(bvh, torch.from_numpy(rays).cuda(), params=params)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.uint32)


def same(got, exp, what):
    e = np.ascontiguousarray(exp).view(np.uint32).reshape(-1, 4)
    bad = np.where(np.any(got != e, axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} of {len(e)} rays differ, first {bad[:5]}"


@pytest.mark.parametrize("kw", LAYOUTS, ids=lambda kw: "-".join(f"{k}={v}" for k, v in kw.items()) or "pbrt")
def test_config1_gpu_built_every_family(sc_mod, oracle_mod, kw):
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    tris = sc.triangles()
    exp = oracle_mod.closest_brute(tris, rays)
    occ = oracle_mod.any_brute(tris, rays)
    bvh = sc_mod.scion_build_gpu(torch.from_numpy(sc.verts).cuda(), sc_mod.layout(**kw),
                                 torch.from_numpy(sc.indices.astype(np.int32)).cuda())
    same(hits(sc_mod, bvh, rays), exp, str(kw))
    same(hits(sc_mod, bvh, rays, dict(rays_per_fetch=1)), exp, str(kw) + " refill")
    assert np.array_equal(occluded(sc_mod, bvh, rays), occ)
    assert sc_mod.scion_get_status(bvh) == 0
    t = sc_mod.scion_bvh_build_times(bvh)
    assert t["logical_ms"] > 0 and t["pack_ms"] >= 0
    if not kw:
        # leaf_max 1: one triangle per leaf, every triangle once; the default
        # (4) collapses subtrees of up to 4 triangles into one leaf
        one = sc_mod.scion_build_gpu(torch.from_numpy(sc.verts).cuda(), sc_mod.layout(leaf_max=1),
                                     torch.from_numpy(sc.indices.astype(np.int32)).cuda())
        assert one.info()["n_nodes"] == 2 * 4096 - 1
        same(hits(sc_mod, one, rays), exp, "leaf_max=1")
        assert bvh.info()["n_nodes"] < 2 * 4096 - 1
        for lm in (2, 8, 15):
            b = sc_mod.scion_build_gpu(torch.from_numpy(sc.verts).cuda(), sc_mod.layout(width=4, leaf_max=lm),
                                       torch.from_numpy(sc.indices.astype(np.int32)).cuda())
            same(hits(sc_mod, b, rays), exp, f"leaf_max={lm}")
            assert np.array_equal(occluded(sc_mod, b, rays), occ)


def test_soup_against_oracle_bvh_and_host_build(sc_mod, oracle_mod):
    rng = scenes.rng_for(41)
    n = 1 << 17
    verts = scenes.random_soup(rng, n, mu=math.log(0.002 * math.sqrt((1 << 23) / n)))
    rays = scenes.random_rays(rng, 1 << 15, (0, 0, 0), (1, 1, 1))
    short = rays.copy()
    short[:, 7] = 0.05
    ob = oracle_mod.BVH2(verts.reshape(-1, 9))
    exp, eocc = ob.closest(rays), ob.any(short)
    d_verts = torch.from_numpy(verts).cuda()
    for kw in (dict(width=4, box_layout="soa", prim_ref="direct"), dict(width=8, box_prec="u8", prim_ref="direct"),
               dict(box_prec="q16", prim_ref="direct")):
        bvh = sc_mod.scion_build_gpu(d_verts, sc_mod.layout(**kw))
        same(hits(sc_mod, bvh, rays), exp, str(kw))
        assert np.array_equal(occluded(sc_mod, bvh, short), eocc), kw
        # a second build gives the same tree
        again = sc_mod.scion_build_gpu(d_verts, sc_mod.layout(**kw))
        assert again.info() == bvh.info()


def test_degenerate_inputs(sc_mod, oracle_mod):
    rng = np.random.default_rng(3)
    # 600 copies of one triangle (all Morton codes equal) plus 60 tiny ones around it
    base = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    off = np.concatenate([rng.uniform(-0.5, 0.5, (60, 1, 2)), rng.uniform(-0.5, -0.1, (60, 1, 1))], axis=2)
    tri = np.concatenate([np.tile(base, (600, 1)), (base[None] * 0.01 + off).reshape(-1, 3)]).astype(np.float32)
    rays = scenes.random_rays(rng, 4096, (-0.5, -0.5, -0.5), (1, 1, 1))
    bvh = sc_mod.scion_build_gpu(torch.from_numpy(tri).cuda(), sc_mod.layout(width=4))
    same(hits(sc_mod, bvh, rays), oracle_mod.closest_brute(tri.reshape(-1, 9), rays), "ties")
    down = np.tile(np.array([[0.25, 0.25, 1.0, 0.0, 0, 0, -1, np.inf]], np.float32), (1, 1))
    h = hits(sc_mod, bvh, down)
    assert h[0, 3] == 0  # equal t on 600 duplicates: lowest id
    # non-finite vertices are left out
    bad = tri.copy()
    bad[3] = np.nan
    bad[10] = np.inf
    b2 = sc_mod.scion_build_gpu(torch.from_numpy(bad).cuda(), sc_mod.layout(width=8, box_prec="u8"))
    same(hits(sc_mod, b2, rays), oracle_mod.closest_brute(bad.reshape(-1, 9), rays), "nonfinite")
    # one triangle, and a scene without a finite triangle
    one = sc_mod.scion_build_gpu(torch.from_numpy(base).cuda(), sc_mod.layout())
    assert hits(sc_mod, one, down)[0, 3] == 0
    nanv = torch.full((9, 3), float("nan"), device="cuda")
    none = sc_mod.scion_build_gpu(nanv, sc_mod.layout(width=4))
    assert np.all(hits(sc_mod, none, rays[:64])[:, 3] == 0xFFFFFFFF)
    assert np.all(occluded(sc_mod, none, rays[:64]) == 0)


def test_invalid_arguments(sc_mod):
    base = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    L = sc_mod.lib()
    h = ctypes.c_void_p()
    d = sc_mod.layout()
    # host memory is rejected
    st = L.scion_build_gpu(base.ctypes.data_as(ctypes.c_void_p), 3, None, 1, ctypes.byref(d), None, ctypes.byref(h))
    assert st == 1 and not h.value
    # an index out of range is rejected before any kernel reads through it
    with pytest.raises(sc_mod.ScionError):
        sc_mod.scion_build_gpu(torch.from_numpy(base).cuda(), d, np.array([[0, 1, 7]], np.uint32))
    with pytest.raises(sc_mod.ScionError):
        sc_mod.scion_build_gpu(torch.from_numpy(base).cuda(), sc_mod.layout(box_prec="q16", leaf_max=16))


def _same_bytes(scion, a, b, what):
    ia, ib = scion.scion_bvh_info(a), scion.scion_bvh_info(b)
    assert ia == ib, f"{what}: info {ia} vs {ib}"
    for name, x, y in zip(("nodes", "nodes2", "prims"), scion.scion_debug_bvh_bytes(a), scion.scion_debug_bvh_bytes(b)):
        assert x.size == y.size, f"{what}: {name} sizes {x.size} vs {y.size}"
        bad = np.flatnonzero(x != y)
        assert bad.size == 0, f"{what}: {name} differ at {bad.size} bytes, first {bad[:8]}"


def test_gpu_packer_bytes_equal_host_packer(sc_mod):
    """The GPU packer writes the same bytes as the host packers for the same
    GPU-built logical tree, on every layout of the test sweep (the treelet
    order and the shared slab are packed on the host by both calls), on an
    indexed height field and on a soup with ties and non-finite triangles."""
    from layout_cases import all_layouts
    scion = sc_mod
    sc = scenes.config1_scene()
    rng = scenes.rng_for(51)
    soup = scenes.random_soup(rng, 3000, mu=math.log(0.05))
    soup[30:33] = soup[0:3]                    # a duplicate triangle: equal Morton codes
    soup[100, 1] = np.nan                      # left out of the tree
    inputs = [(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.indices.astype(np.int32)).cuda()),
              (torch.from_numpy(soup).cuda(), None)]
    for kw in all_layouts():
        for leaf_max in (4, 1):
            desc = scion.layout(leaf_max=leaf_max, **kw)
            for v, ix in inputs:
                try:
                    ref = scion.scion_build_gpu(v, desc, ix, host_pack=True)
                except scion.ScionError as e:  # the layout cannot hold this tree: both must refuse alike
                    with pytest.raises(scion.ScionError) as e2:
                        scion.scion_build_gpu(v, desc, ix)
                    assert e2.value.status == e.status, kw
                    continue
                got = scion.scion_build_gpu(v, desc, ix)
                _same_bytes(scion, got, ref, f"{kw} leaf_max={leaf_max} indexed={ix is not None}")


def test_gpu_packer_full_size(sc_mod, oracle_mod):
    """2^23 random triangles: the GPU packer's bytes equal the host packer's
    for the layouts the benchmark sweeps in both orders and one of each
    own-box codec, and it is much faster than packing on the host."""
    import time
    scion = sc_mod
    sc = scenes.config3_scene()
    dv = torch.from_numpy(sc.verts).cuda()
    for kw in (dict(width=4, box_layout="soa", box_prec="u8", order="bfs", prim_ref="direct"),
               dict(width=4, box_layout="soa", prim_ref="direct"), dict(width=8, box_prec="u8"),
               dict(width=8, box_layout="soa", box_prec="f16", child_ref="indirect", order="bfs"),
               dict(box_prec="q16", box_layout="soa"), dict(prim_ref="direct"),
               dict(box_prec="eq10", child_ref="indirect", order="bfs")):
        desc = scion.layout(**kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = scion.scion_build_gpu(dv, desc)
        t_gpu = time.perf_counter() - t0
        t0 = time.perf_counter()
        ref = scion.scion_build_gpu(dv, desc, host_pack=True)
        t_host = time.perf_counter() - t0
        _same_bytes(scion, got, ref, str(kw))
        assert t_gpu < t_host, (kw, t_gpu, t_host)
        del got, ref
