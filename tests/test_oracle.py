"""Pins for the CPU oracle: closed forms, invariants, exact-arithmetic checks,
brute force against the independent BVH2, and the FP64 gradient against
central differences and exact invariances. No GPU needed."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2511_15028_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TRI0 = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)


def _parse(v):
    return float("inf") if v == "inf" else float(v)


def load_closed_form():
    rows = []
    with open(os.path.join(GOLDEN, "closed_form_hits.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            ray = [_parse(x) for x in lhs.split()]
            rhs = rhs.split()
            exp = None if rhs[0] == "miss" else tuple(float(x) for x in rhs[1:4])
            rows.append((ray, exp))
    return rows


@pytest.mark.parametrize("ray,exp", load_closed_form())
def test_closed_form_single_triangle(oracle_mod, ray, exp):
    got = oracle_mod.intersect(np.array(ray, np.float32), TRI0)
    assert got == exp
    # brute force and BVH2 agree with the single-triangle answer
    r = np.array([ray], np.float32)
    h = oracle_mod.closest_brute(TRI0[None], r)[0]
    b = oracle_mod.BVH2(TRI0[None]).closest(r)[0]
    if exp is None:
        assert h["prim"] == oracle_mod.MISS and np.isinf(h["t"]) and h["u"] == 0 and h["v"] == 0
    else:
        assert h["prim"] == 0 and (h["t"], h["u"], h["v"]) == exp
    assert b.tobytes() == h.tobytes()


def _quad(z=0.0, x0=0.0, y0=0.0, s=1.0):
    a = [x0, y0, z]
    b = [x0 + s, y0, z]
    c = [x0 + s, y0 + s, z]
    d = [x0, y0 + s, z]
    return np.array([a + b + c, a + c + d], np.float32)


def test_shared_edge_tie_goes_to_lowest_id(oracle_mod):
    tris = _quad()
    # ray exactly on the diagonal: both triangles report the same t
    ray = np.array([[0.25, 0.25, 1, 1e-4, 0, 0, -1, np.inf]], np.float32)
    a = oracle_mod.intersect(ray[0], tris[0])
    b = oracle_mod.intersect(ray[0], tris[1])
    assert a is not None and b is not None and a[0] == b[0]
    h = oracle_mod.closest_brute(tris, ray)[0]
    assert h["prim"] == 0
    h2 = oracle_mod.closest_brute(tris[::-1].copy(), ray)[0]
    assert h2["prim"] == 0
    for t in (tris, tris[::-1].copy()):
        assert oracle_mod.BVH2(t, leaf_max=1).closest(ray)[0]["prim"] == 0


def test_duplicate_coplanar_triangles_lowest_id(oracle_mod):
    rng = np.random.default_rng(5)
    tris = np.repeat(TRI0[None], 9, axis=0)
    rays = scenes.make_rays(
        np.stack([rng.uniform(0.05, 0.4, 256), rng.uniform(0.05, 0.4, 256), np.ones(256)], -1).astype(np.float32),
        np.tile(np.array([[0, 0, -1]], np.float32), (256, 1)), 1e-4, np.inf)
    h = oracle_mod.closest_brute(tris, rays)
    assert (h["prim"] == 0).all()
    b = oracle_mod.BVH2(tris, leaf_max=1).closest(rays)
    assert (b["prim"] == 0).all()


def test_fan_vertex_and_closed_mesh_watertight(oracle_mod):
    # six triangles around the origin: a ray through the shared vertex hits
    ang = np.arange(7) * (2 * math.pi / 6)
    fan = []
    for k in range(6):
        fan.append([0, 0, 0, math.cos(ang[k]), math.sin(ang[k]), 0,
                    math.cos(ang[k + 1]), math.sin(ang[k + 1]), 0])
    fan = np.array(fan, np.float32)
    ray = np.array([[0, 0, 1, 1e-4, 0, 0, -1, np.inf]], np.float32)
    hit_count = sum(oracle_mod.intersect(ray[0], f) is not None for f in fan)
    assert hit_count >= 1
    assert oracle_mod.closest_brute(fan, ray)[0]["t"] == 1.0
    # closed icosphere: every ray from inside hits, including rays aimed
    # exactly at vertices and edge midpoints
    v, f = scenes.icosphere(3)
    tris = v[f].reshape(-1, 9).astype(np.float32)
    rng = np.random.default_rng(7)
    dirs = np.concatenate([v, (v[f[:, 0]] + v[f[:, 1]]) / 2, rng.normal(size=(4000, 3))])
    dirs = (dirs / np.linalg.norm(dirs, axis=1, keepdims=True)).astype(np.float32)
    origins = rng.uniform(-0.1, 0.1, size=(dirs.shape[0], 3)).astype(np.float32)
    origins[: v.shape[0] * 2] = 0
    rays = scenes.make_rays(origins, dirs, 0.0, np.inf)
    h = oracle_mod.closest_brute(tris, rays)
    assert (h["prim"] != oracle_mod.MISS).all()


def test_stack_of_parallel_quads_nearest(oracle_mod):
    rng = np.random.default_rng(11)
    quads = np.concatenate([_quad(z=k / 8.0) for k in range(100)])
    perm = rng.permutation(quads.shape[0])
    tris = quads[perm]
    rays = scenes.make_rays(
        np.stack([rng.integers(1, 64, 500) / 64.0, rng.integers(1, 64, 500) / 64.0,
                  np.full(500, 20.0)], -1).astype(np.float32),
        np.tile(np.array([[0, 0, -1]], np.float32), (500, 1)), 1e-4, np.inf)
    h = oracle_mod.closest_brute(tris, rays)
    top = {int(np.where(perm == 198)[0][0]), int(np.where(perm == 199)[0][0])}
    assert np.all(h["t"] == np.float32(20.0 - 99 / 8.0))
    assert set(h["prim"].tolist()) <= top
    b = oracle_mod.BVH2(tris).closest(rays)
    assert b.tobytes() == h.tobytes()


def _exact_inside(o, d, p):
    """Exact rational test of the line o + t d against the triangle: the three
    signed volumes U, V, W (edge functions) and whether they share a strict
    sign. Returns (inside, t, u, v, cond) with t, u, v exact and cond =
    sum of |product terms| / |U + V + W| (the conditioning of u, v)."""
    O = [Fraction(float(x)) for x in o]
    D = [Fraction(float(x)) for x in d]
    P = [[Fraction(float(p[3 * j + k])) for k in range(3)] for j in range(3)]

    def sub(a, b):
        return [a[i] - b[i] for i in range(3)]

    def cross(a, b):
        return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]

    def dot(a, b):
        return sum(a[i] * b[i] for i in range(3))

    A, B, C = sub(P[0], O), sub(P[1], O), sub(P[2], O)
    U = dot(D, cross(C, B))
    V = dot(D, cross(A, C))
    W = dot(D, cross(B, A))
    if not ((U > 0 and V > 0 and W > 0) or (U < 0 and V < 0 and W < 0)):
        return False, None, None, None, None
    det = U + V + W
    n = cross(sub(P[1], P[0]), sub(P[2], P[0]))
    t = dot(n, sub(P[0], O)) / dot(n, D)
    nrm = lambda x: math.sqrt(sum(float(c) ** 2 for c in x))
    mag = nrm(D) * (nrm(C) * nrm(B) + nrm(A) * nrm(C) + nrm(B) * nrm(A))
    return True, t, V / det, W / det, mag / abs(float(det))


def test_intersector_against_exact_rational_arithmetic(oracle_mod):
    """Away from edges, on well-conditioned cases, the float test accepts and
    its t, u, v are within rounding of the exact values (catches dropped terms,
    swapped weights, sign slips)."""
    rng = np.random.default_rng(3)
    n_checked = 0
    for _ in range(800):
        p = rng.normal(size=9).astype(np.float32)
        o = rng.normal(size=3).astype(np.float32) * 3
        target = (p[0:3] * 0.3 + p[3:6] * 0.3 + p[6:9] * 0.4).astype(np.float64)
        jitter = rng.normal(size=3) * rng.choice([0.0, 0.5, 2.0])
        d = (target + jitter - o)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        ray = np.concatenate([o, [-np.inf], d, [np.inf]]).astype(np.float32)
        inside, t, u, v, cond = _exact_inside(o, d, p)
        got = oracle_mod.intersect(ray, p)
        if not inside or cond > 100 or float(t) <= 0:
            continue
        if min(float(u), float(v), 1 - float(u) - float(v)) < 1e-5 * cond:
            continue
        n_checked += 1
        assert got is not None
        tg, ug, vg = got
        scale = float(np.abs(p.reshape(3, 3) - o).max())
        assert abs(tg - float(t)) <= 1e-5 * cond * scale
        assert abs(ug - float(u)) <= 1e-6 * cond
        assert abs(vg - float(v)) <= 1e-6 * cond
    assert n_checked > 200


def test_intersector_exact_miss_agreement(oracle_mod):
    """Rays whose exact crossing is clearly outside the triangle are misses."""
    rng = np.random.default_rng(4)
    for _ in range(400):
        p = rng.normal(size=9).astype(np.float32)
        o = (rng.normal(size=3) * 3).astype(np.float32)
        d = rng.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        ray = np.concatenate([o, [-np.inf], d, [np.inf]]).astype(np.float32)
        P = p.astype(np.float64).reshape(3, 3)
        tuv = oracle_mod.plane_tuv(o, d, P[0], P[1], P[2])
        if tuv is None:
            continue
        t, u, v = tuv
        w = 1 - u - v
        if min(u, v, w) < -1e-3:
            assert oracle_mod.intersect(ray, p) is None
        elif min(u, v, w) > 1e-3 and t < -1e-3:
            assert oracle_mod.intersect(ray, p) is None  # behind the origin
        elif min(u, v, w) > 1e-3 and t > 1e-3:
            got = oracle_mod.intersect(ray, p)
            assert got is not None
            assert abs(got[0] - t) <= 1e-4 * max(1.0, abs(t))


def test_nonfinite_and_degenerate_inputs_miss(oracle_mod):
    ray = np.array([0.25, 0.25, 1, 1e-4, 0, 0, -1, np.inf], np.float32)
    for bad in (np.nan, np.inf, -np.inf):
        t = TRI0.copy()
        t[4] = bad
        assert oracle_mod.intersect(ray, t) is None
    assert oracle_mod.intersect(ray, np.zeros(9, np.float32)) is None  # point triangle
    r = ray.copy()
    r[4:7] = 0  # zero direction
    assert oracle_mod.intersect(r, TRI0) is None
    r = ray.copy()
    r[0] = np.nan
    assert oracle_mod.intersect(r, TRI0) is None
    r = ray.copy()
    r[3], r[7] = 2.0, 1.0  # tmin > tmax
    assert oracle_mod.intersect(r, TRI0) is None
    # a non-finite triangle among good ones is ignored by both traversals
    tris = np.stack([TRI0, TRI0 + np.float32(np.nan)])
    rr = ray[None]
    assert oracle_mod.closest_brute(tris, rr)[0]["prim"] == 0
    assert oracle_mod.BVH2(tris).closest(rr)[0]["prim"] == 0


def _check_invariants(oracle_mod, tris, rays, hits, occ):
    hit = hits["prim"] != oracle_mod.MISS
    t = hits["t"]
    assert np.all(t[hit] >= rays[hit, 3]) and np.all(t[hit] <= rays[hit, 7])
    assert np.all(np.isinf(t[~hit])) and np.all(hits["u"][~hit] == 0) and np.all(hits["v"][~hit] == 0)
    assert np.array_equal(occ.astype(bool), hit)
    u = hits["u"][hit].astype(np.float64)
    v = hits["v"][hit].astype(np.float64)
    assert np.all(u >= 0) and np.all(v >= 0) and np.all(u + v <= 1 + 1e-6)
    # the hit point o + t d lies on the triangle's plane (relative to scale)
    P = tris[hits["prim"][hit]].astype(np.float64).reshape(-1, 3, 3)
    o = rays[hit, 0:3].astype(np.float64)
    d = rays[hit, 4:7].astype(np.float64)
    x = o + t[hit, None].astype(np.float64) * d
    bary = (1 - u - v)[:, None] * P[:, 0] + u[:, None] * P[:, 1] + v[:, None] * P[:, 2]
    scale = np.abs(P).max(axis=(1, 2)) + np.abs(o).max(axis=1) + t[hit]
    assert np.all(np.linalg.norm(x - bary, axis=1) <= 1e-4 * scale)


def test_config1_brute_equals_bvh2_all_rays(oracle_mod):
    sc = scenes.config1_scene()
    tris = sc.triangles()
    rays = scenes.config1_rays()
    assert tris.shape[0] == 4096 and rays.shape[0] == 16384
    bf = oracle_mod.closest_brute(tris, rays)
    bvh = oracle_mod.BVH2(tris, bins=32, leaf_max=4)
    bv = bvh.closest(rays)
    assert bv.tobytes() == bf.tobytes()
    occ_b = oracle_mod.any_brute(tris, rays)
    occ_v = bvh.any(rays)
    assert np.array_equal(occ_b, occ_v)
    assert (bf["prim"] != oracle_mod.MISS).mean() > 0.3
    _check_invariants(oracle_mod, tris, rays, bf, occ_b)
    st = bvh.stats()
    assert st["leaf_tris"] == 4096


def test_soup_and_heightfield_samples_brute_equals_bvh2(oracle_mod):
    rng = scenes.rng_for(77)
    soup = scenes.Scene(scenes.random_soup(rng, 1 << 15, mu=math.log(0.002 * 16)), None)
    tris = soup.triangles()
    rays = scenes.random_rays(rng, 2048, (0, 0, 0), (1, 1, 1))
    bf = oracle_mod.closest_brute(tris, rays)
    bvh = oracle_mod.BVH2(tris)
    assert bvh.closest(rays).tobytes() == bf.tobytes()
    short = rays.copy()
    short[:, 7] = 0.05
    occ = oracle_mod.any_brute(tris, short)
    assert np.array_equal(bvh.any(short), occ)
    _check_invariants(oracle_mod, tris, rays, bf, oracle_mod.any_brute(tris, rays))
    assert 0.05 < occ.mean() < 0.95
    # small fBm height field with spheres, primary + bounce + shadow rays
    sc = scenes.config2_scene(side=65, n_spheres=8)
    tris = sc.triangles()
    prim = scenes.config2_primary(64, 36)
    bvh = oracle_mod.BVH2(tris)
    h = bvh.closest(prim)
    assert h.tobytes() == oracle_mod.closest_brute(tris, prim).tobytes()
    b = scenes.bounce_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"], seed=9)
    s = scenes.shadow_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"])
    assert bvh.closest(b).tobytes() == oracle_mod.closest_brute(tris, b).tobytes()
    assert np.array_equal(bvh.any(s), oracle_mod.any_brute(tris, s))


def test_gradient_closed_form(oracle_mod):
    """Triangle in z = 0, vertical ray o = (x, y, h), d = (0, 0, -1): t = h,
    u = x, v = y, so dL/do = (gu, gv, gt), dL/dd = h (gu, gv, gt), and moving
    p0 along z by e changes t by -e (1 - x - y) while u, v stay fixed."""
    x, y, h = 0.25, 0.125, 2.0
    ray = np.array([[x, y, h, 1e-4, 0, 0, -1, np.inf]], np.float32)
    hits = oracle_mod.closest_brute(TRI0[None], ray)
    g = np.array([[0.5, -1.5, 2.0]], np.float32)
    gv, gr = oracle_mod.grad(TRI0[None], None, 3, ray, hits, g)
    gt, gu, gvv = g[0]
    np.testing.assert_allclose(gr[0, :3], [gu, gvv, gt], rtol=0, atol=1e-12)
    np.testing.assert_allclose(gr[0, 3:], [h * gu, h * gvv, h * gt], rtol=0, atol=1e-12)
    assert abs(gv[0, 2] - (-gt * (1 - x - y))) < 1e-12
    assert abs(gv[1, 2] - (-gt * x)) < 1e-12
    assert abs(gv[2, 2] - (-gt * y)) < 1e-12


def test_gradient_invariances_and_fd_config1(oracle_mod):
    sc = scenes.config1_scene()
    tris = sc.triangles()
    rays = scenes.config1_rays()
    hits = oracle_mod.BVH2(tris).closest(rays)
    w, a, b = scenes.config5_weights(rays.shape[0])
    g = np.stack([w, a, b], -1)
    nv = sc.verts.shape[0]
    gv, gr = oracle_mod.grad(tris, sc.indices, nv, rays, hits, g)
    fv, fr = oracle_mod.grad_fd(tris, sc.indices, nv, rays, hits, g, 1e-3)
    hit = hits["prim"] != oracle_mod.MISS
    # translation invariance per ray: dL/do + sum_j dL/dp_j = 0
    sub_hits = hits[hit][:50].copy()
    sub_hits["prim"] = np.arange(50)
    gv1, gr1 = oracle_mod.grad(tris[hits["prim"][hit][:50]], None, 150, rays[hit][:50], sub_hits, g[hit][:50])
    per_ray_p = gv1.reshape(50, 3, 3).sum(axis=1)
    np.testing.assert_allclose(per_ray_p + gr1[:, :3], 0, atol=1e-9)
    # scale homogeneity: d . dL/dd = -g_t t
    d = rays[hit][:50, 4:7].astype(np.float64)
    lhs = (d * gr1[:, 3:]).sum(axis=1)
    np.testing.assert_allclose(lhs, -g[hit][:50, 0].astype(np.float64) * sub_hits["t"].astype(np.float64), rtol=1e-9, atol=1e-9)
    # central differences converge to the analytic FP64 gradient: the
    # truncation error of the h = 1e-3 differences is O((h/L)^2) for triangles
    # of size L ~ 0.03, and shrinks 100-fold at h = 1e-4
    scale = np.abs(gv).max()
    rscale = np.abs(gr).max()
    np.testing.assert_allclose(fv, gv, rtol=0, atol=1e-2 * scale)
    np.testing.assert_allclose(fr[hit], gr[hit], rtol=0, atol=1e-2 * rscale)
    fv4, fr4 = oracle_mod.grad_fd(tris, sc.indices, nv, rays, hits, g, 1e-4)
    np.testing.assert_allclose(fv4, gv, rtol=0, atol=1e-4 * scale)
    np.testing.assert_allclose(fr4[hit], gr[hit], rtol=0, atol=1e-4 * rscale)
    assert np.abs(fv4 - gv).max() < 0.05 * np.abs(fv - gv).max()
    assert np.all(gr[~hit] == 0)


# ------------------------------------------------------------------ closest point query
def _seg_point_f64(p, a, b):
    ab = b - a
    den = ab @ ab
    s = 0.0 if den == 0.0 else min(1.0, max(0.0, ((p - a) @ ab) / den))
    return a + s * ab


def _dist_f64(p, tri):
    """Distance from p to a triangle in float64 by another method than the
    oracle's: the plane projection if it falls inside the triangle
    (barycentrics from normal equations), else the nearest of the three
    clamped edge projections."""
    a, b, c = (np.asarray(tri[3 * k:3 * k + 3], np.float64) for k in range(3))
    p = np.asarray(p, np.float64)
    e1, e2 = b - a, c - a
    G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
    cands = [_seg_point_f64(p, a, b), _seg_point_f64(p, a, c), _seg_point_f64(p, b, c)]
    if abs(np.linalg.det(G)) > 1e-12 * (e1 @ e1) * (e2 @ e2) + 1e-300:
        s, t = np.linalg.solve(G, np.array([(p - a) @ e1, (p - a) @ e2]))
        if s >= 0 and t >= 0 and s + t <= 1:
            cands.append(a + s * e1 + t * e2)
    return min(np.linalg.norm(p - q) for q in cands)


@pytest.mark.parametrize("pt,exp", [
    ((0.25, 0.25, 2.0), (4.0, 0.25, 0.25)),     # face: straight above the interior
    ((-1.0, -1.0, 0.0), (2.0, 0.0, 0.0)),       # vertex p0
    ((2.0, -1.0, 0.0), (2.0, 1.0, 0.0)),        # vertex p1
    ((-0.5, 3.0, 0.0), (4.25, 0.0, 1.0)),       # vertex p2
    ((0.5, -1.0, 0.0), (1.0, 0.5, 0.0)),        # edge p0p1
    ((-1.0, 0.5, 3.0), (10.0, 0.0, 0.5)),       # edge p0p2
    ((1.0, 1.0, 0.0), (0.5, 0.5, 0.5)),         # edge p1p2
    ((0.25, 0.5, 0.0), (0.0, 0.25, 0.5)),       # on the triangle
])
def test_closest_point_closed_forms(oracle_mod, pt, exp):
    """Dyadic cases in every Voronoi region of (0,0,0), (1,0,0), (0,1,0):
    exact squared distance and barycentric weights of p1, p2."""
    tri = [0, 0, 0, 1, 0, 0, 0, 1, 0]
    assert oracle_mod.closest_point(pt, tri) == exp


def test_closest_point_against_independent_f64(oracle_mod):
    """Random triangles (including slivers and near-degenerate ones) and points
    at several distances: the f32 result is within f32 rounding of the
    float64 distance computed by another method, the weights lie in the
    triangle, and they rebuild a point at that distance."""
    rng = np.random.default_rng(11)
    n_bad = 0
    for i in range(3000):
        tri = rng.normal(size=9) * (10.0 ** rng.uniform(-3, 2))
        if i % 10 == 0:
            tri[6:9] = tri[0:3] + (tri[3:6] - tri[0:3]) * rng.uniform(0, 1) + rng.normal(size=3) * 1e-4
        tri = tri.astype(np.float32)
        p = (tri[:3] + rng.normal(size=3) * (10.0 ** rng.uniform(-4, 2))).astype(np.float32)
        d2, u, v = oracle_mod.closest_point(p, tri)
        ref = _dist_f64(p, tri.astype(np.float64))
        scale = float(np.abs(np.concatenate([tri, p])).max())
        assert abs(math.sqrt(d2) - ref) <= 1e-5 * (ref + scale), (i, d2, ref * ref)
        assert u >= 0 and v >= 0 and u + v <= 1 + 1e-6
        a, b, c = (tri[3 * k:3 * k + 3].astype(np.float64) for k in range(3))
        q = (1 - u - v) * a + u * b + v * c
        n_bad += abs(np.linalg.norm(p - q) - math.sqrt(d2)) > 1e-4 * (ref + scale)
    assert n_bad == 0


def test_closest_point_degenerate_and_nonfinite(oracle_mod):
    # a triangle collapsed to a segment, and to a point
    seg = [0, 0, 0, 2, 0, 0, 1, 0, 0]
    assert oracle_mod.closest_point((1.0, 3.0, 0.0), seg)[0] == 9.0
    assert oracle_mod.closest_point((-2.0, 0.0, 0.0), seg)[0] == 4.0
    pt = [1, 1, 1] * 3
    assert oracle_mod.closest_point((1.0, 1.0, 3.0), pt)[0] == 4.0
    assert oracle_mod.closest_point((0.0, 0.0, 0.0), [0, 0, 0, 1, 0, 0, float("nan"), 1, 0]) is None


def test_cpq_brute_ties_radius_and_miss(oracle_mod):
    """Lowest id among equal distances; only triangles with d2 <= r2max
    count (closed); a point with a non-finite coordinate or an empty scene
    gives a miss."""
    base = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)
    far = base + np.array([0, 0, 5] * 3, np.float32)
    tris = np.stack([far, base, base, far])
    pts = np.array([[0.25, 0.25, 1.0, np.inf],   # nearest: the two copies of base, d2 = 1
                    [0.25, 0.25, 1.0, 1.0],       # radius exactly 1: still found
                    [0.25, 0.25, 1.0, 0.99],      # radius below: miss
                    [0.25, 0.25, 4.0, np.inf],    # nearer to the far copies: id 0
                    [np.nan, 0.0, 0.0, np.inf],   # a point that is not finite: miss
                    [np.inf, 0.0, 0.0, np.inf]], np.float32)
    out = oracle_mod.cpq_brute(tris, pts)
    assert list(out["prim"]) == [1, 1, 0xFFFFFFFF, 0, 0xFFFFFFFF, 0xFFFFFFFF]
    assert out["t"][0] == 1.0 and out["t"][3] == 1.0 and math.isinf(out["t"][2])
    assert out["u"][0] == 0.25 and out["v"][0] == 0.25
    empty = oracle_mod.cpq_brute(np.zeros((0, 9), np.float32), pts[:1])
    assert empty["prim"][0] == 0xFFFFFFFF


def test_cpq_brute_is_the_minimum_over_triangles(oracle_mod):
    """On a soup, the brute force equals the minimum of the single-triangle
    evaluations (lexicographic in (d2, id))."""
    rng = np.random.default_rng(5)
    tris = scenes.random_soup(rng, 300, mu=math.log(0.05)).reshape(-1, 9)
    pts = np.concatenate([rng.uniform(-0.2, 1.2, (64, 3)), np.full((64, 1), np.inf)], 1).astype(np.float32)
    out = oracle_mod.cpq_brute(tris, pts)
    for j in range(64):
        d = [oracle_mod.closest_point(pts[j, :3], t)[0] for t in tris]
        k = min(range(len(d)), key=lambda i: (d[i], i))
        assert out["prim"][j] == k and out["t"][j] == d[k]
