"""GPU closest point query (App. G) on every layout: results (d2, u, v, prim)
bit-identical to the CPU oracle's brute force, with search radii, points on
and far from the surface, non-finite points, refit trees and the counting
variant."""
import math

import numpy as np
import pytest

from layout_cases import all_layouts
from paper_2511_15028_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = [kw for kw in all_layouts() if kw["box_prec"] != "slab"]  # slab: no CPQ


@pytest.fixture(scope="module")
def sc_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15028_gb300 import build as b
    b.build()
    from paper_2511_15028_gb300 import scion
    scion.lib()
    return scion


def points_around(verts, n, seed, margin=0.3, r2=np.inf):
    rng = np.random.default_rng(seed)
    lo, hi = verts.min(0) - margin, verts.max(0) + margin
    p = lo + (hi - lo) * rng.uniform(size=(n, 3))
    return np.concatenate([p, np.full((n, 1), r2)], 1).astype(np.float32)


def query(scion, bvh, pts, params=None):
    out = scion.scion_query_closest_point(bvh, torch.from_numpy(pts).cuda(), params=params)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).reshape(-1, 4)


def same(got, exp, what):
    e = np.ascontiguousarray(exp).view(np.uint32).reshape(-1, 4)
    bad = np.where(np.any(got != e, axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} of {len(e)} points differ, first {bad[:5]}: {got[bad[:2]]} vs {e[bad[:2]]}"


@pytest.fixture(scope="module")
def config1_points(oracle_mod):
    sc = scenes.config1_scene()
    pts = points_around(sc.verts, 8192, 101)
    return sc, pts, oracle_mod.cpq_brute(sc.triangles(), pts)


@pytest.mark.parametrize("kw", ALL, ids=lambda kw: "-".join(str(v) for v in kw.values()))
def test_config1_every_layout(sc_mod, config1_points, kw):
    sc, pts, exp = config1_points
    bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(**kw), sc.indices)
    same(query(sc_mod, bvh, pts), exp, str(kw))
    same(query(sc_mod, bvh, pts, dict(ordered_children=2)), exp, str(kw) + " slot order")
    assert sc_mod.scion_get_status(bvh) == 0


def test_radius_surface_far_and_nonfinite_points(sc_mod, oracle_mod):
    sc = scenes.config1_scene()
    tris = sc.triangles()
    rng = np.random.default_rng(7)
    # points on the surface (a vertex or an interior point of a triangle)
    k = rng.integers(0, tris.shape[0], 512)
    w = rng.dirichlet([1, 1, 1], 512)
    on = np.einsum("ij,ijk->ik", w, tris[k].reshape(-1, 3, 3))
    surf = np.concatenate([on, np.zeros((512, 1))], 1)
    verts = np.concatenate([sc.verts[:256], np.full((256, 1), np.inf)], 1)
    far = points_around(sc.verts, 256, 8, margin=1e3)
    radius = points_around(sc.verts, 1024, 9)
    radius[:, 3] = rng.uniform(0, 0.05, 1024) ** 2
    bad = np.array([[np.nan, 0, 0, np.inf], [np.inf, 0, 0, np.inf], [0, 0, 0, np.nan], [0, 0, 0, -1.0]])
    pts = np.concatenate([surf, verts, far, radius, bad]).astype(np.float32)
    exp = oracle_mod.cpq_brute(tris, pts)
    assert (exp["prim"] == 0xFFFFFFFF).sum() >= 4
    for kw in (dict(), dict(width=4, box_layout="soa", prim_ref="direct"), dict(width=8, box_prec="u8"),
               dict(width=8, box_prec="f16", box_layout="soa"), dict(box_prec="q16"), dict(box_prec="eq10")):
        bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(**kw), sc.indices)
        same(query(sc_mod, bvh, pts), exp, str(kw))


def test_soup_gpu_built_refit_and_counting(sc_mod, oracle_mod):
    rng = scenes.rng_for(51)
    n = 1 << 16
    soup = scenes.random_soup(rng, n, mu=math.log(0.002 * math.sqrt((1 << 23) / n)))
    pts = points_around(soup, 4096, 52, margin=0.1)
    exp = oracle_mod.cpq_brute(soup.reshape(-1, 9), pts)
    for kw in (dict(width=4, box_layout="soa", prim_ref="direct"), dict(width=8, box_prec="u8", prim_ref="direct"),
               dict(box_prec="q16", prim_ref="direct")):
        bvh = sc_mod.scion_build_gpu(torch.from_numpy(soup).cuda(), sc_mod.layout(**kw))
        same(query(sc_mod, bvh, pts), exp, f"gpu-built {kw}")
        out, cnt = sc_mod.scion_trace_stats(bvh, torch.from_numpy(pts).cuda(), 2)
        same(out.cpu().numpy().view(np.uint32).reshape(-1, 4), exp, f"counting {kw}")
        c = cnt.cpu().numpy()
        assert c[3] == pts.shape[0] and c[0] > 0 and c[2] > 0
        moved = (soup + 0.01 * np.sin(soup * 13.0)).astype(np.float32)
        sc_mod.scion_refit(bvh, torch.from_numpy(moved).cuda())
        same(query(sc_mod, bvh, pts), oracle_mod.cpq_brute(moved.reshape(-1, 9), pts), f"refit {kw}")
    with pytest.raises(sc_mod.ScionError):
        query(sc_mod, bvh, pts, dict(rays_per_fetch=1))
    slab = sc_mod.scion_build(soup, sc_mod.layout(box_prec="slab"))
    with pytest.raises(sc_mod.ScionError) as e:
        query(sc_mod, slab, pts)
    assert e.value.status == 2  # unsupported layout


def test_points_in_pinned_host_memory(sc_mod, config1_points):
    """Query points and results in pinned host memory, read and written by the
    kernel in place: the same records as from device buffers."""
    sc, pts, exp = config1_points
    bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(width=4, box_layout="soa"), sc.indices)
    h_pts = torch.from_numpy(pts).pin_memory()
    out = sc_mod.scion_query_closest_point(bvh, h_pts)
    torch.cuda.synchronize()
    assert not out.is_cuda and out.is_pinned()
    same(out.numpy().view(np.uint32).reshape(-1, 4), exp, "pinned points")
