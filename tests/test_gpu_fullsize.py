"""Full-size parity in the launch configuration the benchmark times (default
trace parameters): the coherent+incoherent workload (1,373,138 triangles,
1920x1080 primary rays plus bounce and shadow rays) on all swept layouts, and
the incoherent 2^23-triangle soup with 2^23 random rays (closest hit and
any hit with tmax 0.05). Config-2 outputs are all compared with the CPU
oracle's BVH2 (bounce and shadow rays come from its own primary hits);
config-3 outputs too (all 2^23 rays of both queries), the oracle's BVH2
itself being checked against brute force over all 2^23 triangles on 4,096
sampled rays of each query."""
import numpy as np
import pytest

from paper_2511_15028_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15028_gb300 import build as b
    b.build()
    from paper_2511_15028_gb300 import scion
    scion.lib()
    return scion


def _cmp(scion, got_i32, exp, what):
    g = got_i32.cpu().numpy().view(np.uint32).reshape(-1, 4)
    e = np.ascontiguousarray(exp).view(np.uint32).reshape(-1, 4)
    bad = np.where(np.any(g != e, axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} of {len(e)} differ, e.g. {bad[:5]}"


def test_config2_full_size_all_layouts(sc_mod, oracle_mod):
    scion = sc_mod
    sc = scenes.config2_scene()
    assert sc.n_tris == 1_373_138
    prim = scenes.config2_primary()
    ob = oracle_mod.BVH2(sc.triangles())
    hp = ob.closest(prim)
    bounce = scenes.bounce_rays(sc, prim, hp["t"], hp["u"], hp["v"], hp["prim"], seed=2002)
    shadow = scenes.shadow_rays(sc, prim, hp["t"], hp["u"], hp["v"], hp["prim"])
    hb = ob.closest(bounce)
    hs = ob.any(shadow)
    d = [torch.from_numpy(r).cuda() for r in (prim, bounce, shadow)]
    for name, desc in scion.sweep_layouts(extended=True).items():
        bvh = scion.scion_build(sc.verts, desc, sc.indices)
        _cmp(scion, scion.scion_trace_closest(bvh, d[0]), hp, name + " primary")
        _cmp(scion, scion.scion_trace_closest(bvh, d[1]), hb, name + " bounce")
        occ = scion.scion_trace_any(bvh, d[2]).cpu().numpy().astype(np.uint32)
        assert np.array_equal(occ, hs), name + " shadow"
        assert scion.scion_get_status(bvh) == 0


@pytest.fixture(scope="module")
def config3(oracle_mod):
    """The 2^23-triangle soup and rays with the oracle's answers for every
    ray: its BVH2 traversal over all rays, checked on 4,096 sampled rays of
    each query against brute force over every triangle (the definition)."""
    sc = scenes.config3_scene()
    assert sc.n_tris == 1 << 23
    rays = scenes.config3_rays()
    short = rays.copy()
    short[:, 7] = 0.05
    tris = sc.verts.reshape(-1, 9)
    ob = oracle_mod.BVH2(tris)
    exp = ob.closest(rays)
    eocc = ob.any(short)
    del ob
    pick = np.sort(np.random.default_rng(5).choice(rays.shape[0], 4096, replace=False))
    brute = oracle_mod.closest_brute(tris, rays[pick])
    assert brute.tobytes() == exp[pick].tobytes(), "oracle BVH2 vs brute force (closest)"
    assert np.array_equal(oracle_mod.any_brute(tris, short[pick]), eocc[pick]), "oracle BVH2 vs brute force (any)"
    assert 0.3 < (exp["prim"] != 0xFFFFFFFF).mean() and 0.02 < eocc.mean() < 0.98
    return sc, rays, short, exp, eocc


def test_config3_full_size(sc_mod, config3):
    """Every swept layout (also in breadth-first order) traces all 2^23 rays
    (closest hit, and any hit with tmax 0.05); every result equals the
    oracle's."""
    scion = sc_mod
    sc, rays, short, exp, eocc = config3
    d, ds = torch.from_numpy(rays).cuda(), torch.from_numpy(short).cuda()
    for name, desc in scion.sweep_layouts(extended=True, orders=True).items():
        bvh = scion.scion_build(sc.verts, desc)
        _cmp(scion, scion.scion_trace_closest(bvh, d), exp, name + " closest")
        occ = scion.scion_trace_any(bvh, ds).cpu().numpy().astype(np.uint32)
        bad = np.flatnonzero(occ != eocc)
        assert bad.size == 0, f"{name} any: {bad.size} differ, e.g. {bad[:5]}"
        assert scion.scion_get_status(bvh) == 0
        del bvh


def test_config3_full_size_gpu_built(sc_mod, config3):
    """The 2^23-triangle soup with its logical BVH2 built on the GPU (linear
    BVH), packed as BVH8 u8 and BVH4: all rays against the oracle, also with
    the newest stack entries in registers."""
    scion = sc_mod
    sc, rays, short, exp, eocc = config3
    d, ds = torch.from_numpy(rays).cuda(), torch.from_numpy(short).cuda()
    dv = torch.from_numpy(sc.verts).cuda()
    for desc in (scion.layout(width=8, box_prec="u8", prim_ref="direct"),
                 scion.layout(width=4, box_layout="soa", prim_ref="direct", order="bfs")):
        bvh = scion.scion_build_gpu(dv, desc)
        for p in (None, dict(reg_stack=4, rays_per_fetch=4)):
            _cmp(scion, scion.scion_trace_closest(bvh, d, params=p), exp, f"gpu-built closest {p}")
            occ = scion.scion_trace_any(bvh, ds, params=p).cpu().numpy().astype(np.uint32)
            assert np.array_equal(occ, eocc), f"gpu-built any {p}"
        assert scion.scion_get_status(bvh) == 0
        del bvh


def test_config2_full_size_closest_point(sc_mod, oracle_mod):
    """2^20 query points in the coherent scene's box (the paper's CPQ point
    count) on the swept layouts; 256 sampled points against brute force over
    all 1,373,138 triangles."""
    scion = sc_mod
    sc = scenes.config2_scene()
    rng = np.random.default_rng(2005)
    lo, hi = sc.verts.min(0) - 0.1, sc.verts.max(0) + 0.1
    pts = np.concatenate([lo + (hi - lo) * rng.uniform(size=(1 << 20, 3)), np.full((1 << 20, 1), np.inf)],
                         1).astype(np.float32)
    pick = np.sort(rng.choice(pts.shape[0], 256, replace=False))
    exp = oracle_mod.cpq_brute(sc.triangles(), pts[pick])
    d = torch.from_numpy(pts).cuda()
    for name, desc in scion.sweep_layouts(extended=True).items():
        if name.endswith("indirect") or name.startswith("bvh2_slab"):  # slab: rays only
            continue
        bvh = scion.scion_build(sc.verts, desc, sc.indices)
        got = scion.scion_query_closest_point(bvh, d)[torch.from_numpy(pick).cuda()]
        _cmp(scion, got, exp, name + " closest point")
        assert scion.scion_get_status(bvh) == 0
