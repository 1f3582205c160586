"""GPU parity: every layout's closest-hit and any-hit results match the CPU
oracle bit for bit (hit/miss, prim, t, u, v), through the C ABI."""
import ctypes
import math

import numpy as np
import pytest

from layout_cases import all_layouts
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


def gpu_closest(scion, bvh, rays, params=None):
    r = torch.from_numpy(np.ascontiguousarray(rays, np.float32)).cuda()
    h = scion.scion_trace_closest(bvh, r, params=params)
    torch.cuda.synchronize()
    return scion.split_hits(h)


def gpu_any(scion, bvh, rays, params=None):
    r = torch.from_numpy(np.ascontiguousarray(rays, np.float32)).cuda()
    o = scion.scion_trace_any(bvh, r, params=params)
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.uint32)


def assert_same_hits(got, exp, what=""):
    g = got.view(np.uint32).reshape(-1, 4)
    e = np.ascontiguousarray(exp).view(np.uint32).reshape(-1, 4)
    bad = np.where(np.any(g != e, axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}: gpu {got[bad[:3]]} oracle {exp[bad[:3]]}"


ALL = all_layouts()


@pytest.fixture(scope="module")
def config1(oracle_mod):
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    tris = sc.triangles()
    exp = oracle_mod.closest_brute(tris, rays)
    occ = oracle_mod.any_brute(tris, rays)
    return sc, rays, exp, occ


@pytest.mark.parametrize("kw", ALL, ids=lambda kw: "-".join(str(v) for v in kw.values()))
def test_config1_every_layout_bit_exact(sc_mod, config1, kw):
    sc, rays, exp, occ = config1
    bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(**kw), sc.indices)
    got = gpu_closest(sc_mod, bvh, rays)
    assert_same_hits(got, exp, str(kw))
    assert np.array_equal(gpu_any(sc_mod, bvh, rays), occ)
    unordered = gpu_closest(sc_mod, bvh, rays, params=dict(ordered_children=2))
    assert_same_hits(unordered, exp, "unordered")
    lane = gpu_closest(sc_mod, bvh, rays, params=dict(rays_per_fetch=1))
    assert_same_hits(lane, exp, "refill 1")
    lane = gpu_closest(sc_mod, bvh, rays, params=dict(rays_per_fetch=13))
    assert_same_hits(lane, exp, "refill 13")
    nearest = gpu_closest(sc_mod, bvh, rays, params=dict(ordered_children=3))
    assert_same_hits(nearest, exp, "nearest first")
    # the rays are a 128 x 128 raster: 8x4 pixel tiles per warp; also widths
    # that leave ragged tiles on the right edge and a partial last row
    for w in (128, 100, 7, 1, 1 << 20):
        tiled = gpu_closest(sc_mod, bvh, rays, params=dict(raster_width=w, ordered_children=3))
        assert_same_hits(tiled, exp, f"raster {w}")
        assert np.array_equal(gpu_any(sc_mod, bvh, rays, params=dict(raster_width=w)), occ)
    assert np.array_equal(gpu_any(sc_mod, bvh, rays, params=dict(rays_per_fetch=1)), occ)
    assert np.array_equal(gpu_any(sc_mod, bvh, rays, params=dict(rays_per_fetch=31)), occ)
    # the newest stack entries in registers (2 or 4), spilling to a shared
    # part that is itself tiny (1 entry) or the default, with every fetch mode
    for p in (dict(reg_stack=2), dict(reg_stack=4, rays_per_fetch=1), dict(reg_stack=4, smem_stack=1),
              dict(reg_stack=2, smem_stack=1, rays_per_fetch=8, ordered_children=3),
              dict(reg_stack=4, raster_width=128, ordered_children=2)):
        assert_same_hits(gpu_closest(sc_mod, bvh, rays, params=p), exp, f"{kw} {p}")
        assert np.array_equal(gpu_any(sc_mod, bvh, rays, params=p), occ), f"{kw} {p}"
    assert sc_mod.scion_get_status(bvh) == 0


def test_closed_form_scenes_on_gpu(sc_mod, oracle_mod):
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    quad = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 0, 0], [1, 1, 0], [0, 1, 0]], np.float32)
    rays = []
    for x, y in ((0.25, 0.5), (0.0, 0.0), (1.0, 0.0), (0.5, 0.5), (0.75, 0.5), (0.25, 0.25)):
        rays.append([x, y, 1, 1e-4, 0, 0, -1, np.inf])
    rays += [[0.25, 0.5, 1, 1, 0, 0, -1, np.inf], [0.25, 0.5, 1, 1e-4, 0, 0, -1, 1],
             [0.25, 0.5, 1, 1e-4, 0, 0, -1, 0.5], [0.25, 0.5, 1, 2, 0, 0, -1, 1],
             [0.25, 0.5, 1, 1e-4, 0, 0, 0, np.inf], [0.25, 0.5, 1, 1e-4, 1, 0, 0, np.inf],
             [0.25, 0.5, -1, 1e-4, 0, 0, 1, np.inf], [0.25, 0.5, 1, 1e-4, 0, 0, 1, np.inf]]
    rays = np.array(rays, np.float32)
    for verts in (tri, quad):
        for kw in ALL[::7]:
            bvh = sc_mod.scion_build(verts, sc_mod.layout(**kw))
            exp = oracle_mod.closest_brute(verts.reshape(-1, 9), rays)
            assert_same_hits(gpu_closest(sc_mod, bvh, rays), exp, str(kw))
            assert np.array_equal(gpu_any(sc_mod, bvh, rays), oracle_mod.any_brute(verts.reshape(-1, 9), rays))


def test_ties_duplicates_and_stack_of_quads(sc_mod, oracle_mod):
    rng = np.random.default_rng(11)
    quads = []
    for k in range(100):
        z = k / 8.0
        quads += [[0, 0, z], [1, 0, z], [1, 1, z], [0, 0, z], [1, 1, z], [0, 1, z]]
    verts = np.array(quads, np.float32).reshape(-1, 9)[rng.permutation(200)].reshape(-1, 3)
    dup = np.repeat(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)[None], 9, 0).reshape(-1, 3)
    o = np.stack([rng.integers(1, 64, 4096) / 64.0, rng.integers(1, 64, 4096) / 64.0, np.full(4096, 20.0)], -1)
    rays = scenes.make_rays(o.astype(np.float32), np.tile(np.float32([[0, 0, -1]]), (4096, 1)), 1e-4, np.inf)
    diag = rays.copy()
    diag[:, 1] = diag[:, 0]  # exactly on the quads' shared diagonal: ties
    for v in (verts, dup):
        for kw in ALL[::5]:
            bvh = sc_mod.scion_build(v, sc_mod.layout(**kw))
            for rr in (rays, diag):
                assert_same_hits(gpu_closest(sc_mod, bvh, rr), oracle_mod.closest_brute(v.reshape(-1, 9), rr), str(kw))


def test_edge_cases(sc_mod, oracle_mod):
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    bvh = sc_mod.scion_build(sc.verts, sc_mod.layout())
    # n = 0 is a no-op
    empty = torch.zeros((0, 8), dtype=torch.float32, device="cuda")
    assert sc_mod.scion_trace_closest(bvh, empty).shape == (0, 4)
    # degenerate rays: zero direction, NaN origin, tmin > tmax, axis-parallel
    bad = rays[:64].copy()
    bad[0, 4:7] = 0
    bad[1, 0] = np.nan
    bad[2, 3], bad[2, 7] = 5.0, 1.0
    bad[3, 4:7] = [0, 0, -1]
    bad[4, 4:7] = [0, 0, 1]
    bad[5, 4:7] = [1, 0, 0]
    bad[6, 0:3] = [0.0, 0.0, 0.5]
    bad[6, 4:7] = [0, -1, 0]
    bad[7, 3] = -np.inf  # tmin below zero counts as zero
    bad[8, 3] = np.nan
    bad[9, 0:3] = [0.1, 0.1, -1.0]  # below the surface looking up, tmin < 0
    bad[9, 3] = -10.0
    bad[9, 4:7] = [0, 0, 1]
    exp = oracle_mod.closest_brute(sc.triangles(), bad)
    for kw in ALL[::3]:
        b = sc_mod.scion_build(sc.verts, sc_mod.layout(**kw), sc.indices)
        assert_same_hits(gpu_closest(sc_mod, b, bad), exp, str(kw))
    # scenes with no hittable triangle, and a scene with non-finite triangles
    none = np.full((9, 3), np.nan, np.float32)
    for kw in ({}, dict(width=8, box_prec="u8")):
        b = sc_mod.scion_build(none, sc_mod.layout(**kw))
        got = gpu_closest(sc_mod, b, rays[:100])
        assert np.all(got["prim"] == 0xFFFFFFFF) and np.all(np.isinf(got["t"]))
        assert np.all(gpu_any(sc_mod, b, rays[:100]) == 0)
    v = sc.triangles().reshape(-1, 3).copy()
    v[7] = np.inf
    v[300] = np.nan
    b = sc_mod.scion_build(v, sc_mod.layout(width=4))
    assert_same_hits(gpu_closest(sc_mod, b, rays), oracle_mod.closest_brute(v.reshape(-1, 9), rays), "nonfinite")


def test_device_errors_are_reported_not_faulted(sc_mod):
    """A tiny step limit and a stack deeper than the traversal stack end the
    affected rays with prim = ERROR and a status code; nothing faults."""
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(), sc.indices)
    got = gpu_closest(sc_mod, bvh, rays, params=dict(max_steps=1))
    assert np.any(got["prim"] == 0xFFFFFFFE)
    assert sc_mod.scion_get_status(bvh) == 6
    assert sc_mod.scion_get_status(bvh) == 0  # cleared
    got = gpu_closest(sc_mod, bvh, rays, params=dict(max_steps=1, rays_per_fetch=4))
    assert np.any(got["prim"] == 0xFFFFFFFE) and sc_mod.scion_get_status(bvh) == 6
    with pytest.raises(sc_mod.ScionError):
        gpu_closest(sc_mod, bvh, rays, params=dict(rays_per_fetch=33))
    with pytest.raises(sc_mod.ScionError):  # tiles need warp batches
        gpu_closest(sc_mod, bvh, rays, params=dict(raster_width=128, rays_per_fetch=8))
    # a chain: triangles at x = 4^k (k = -50..49) whose two-bin SAH tree peels
    # one triangle per level (depth 100); a ray along +x through all of them
    # pushes one far child per level, more than the 64-entry stack holds
    n = 100
    c = 4.0 ** (np.arange(n) - n // 2)
    s = c / 2
    v = np.zeros((n, 3, 3))
    v[:, 0] = np.stack([c, -s, -s], -1)
    v[:, 1] = np.stack([c, s, -s], -1)
    v[:, 2] = np.stack([c, 0 * s, 2 * s], -1)
    v = v.astype(np.float32).reshape(-1, 3)
    desc = sc_mod.layout(leaf_max=1, sah_bins=2)
    assert sc_mod.scion_debug_build_host(v, desc).info["depth"] == n
    b = sc_mod.scion_build(v, desc)
    ray = np.array([[-1.0, 0.0, 0.0, 0.0, 1, 0, 0, np.inf]], np.float32)
    got = gpu_closest(sc_mod, b, ray)
    assert got["prim"][0] == 0xFFFFFFFE
    assert sc_mod.scion_get_status(b) == 5
    got = gpu_closest(sc_mod, b, ray, params=dict(rays_per_fetch=1))
    assert got["prim"][0] == 0xFFFFFFFE and sc_mod.scion_get_status(b) == 5
    # four more entries in registers still hold fewer than 100
    got = gpu_closest(sc_mod, b, ray, params=dict(reg_stack=4))
    assert got["prim"][0] == 0xFFFFFFFE and sc_mod.scion_get_status(b) == 5
    for rs in (1, 3, 5, 8):
        with pytest.raises(sc_mod.ScionError):
            gpu_closest(sc_mod, bvh, rays, params=dict(reg_stack=rs))
    with pytest.raises(sc_mod.ScionError):  # closest point queries keep their stack in memory
        sc_mod.scion_query_closest_point(bvh, torch.zeros((32, 4), dtype=torch.float32, device="cuda"),
                                         params=dict(reg_stack=2))
    # a short ray that ends before the deep part is unaffected
    ok = gpu_any(sc_mod, b, np.array([[-1.0, 0.0, 0.0, 0.0, -1, 0, 0, np.inf]], np.float32))
    assert ok[0] == 0 and sc_mod.scion_get_status(b) == 0


def test_config2_reduced_all_ray_kinds(sc_mod, oracle_mod):
    """Scaled-down coherent + incoherent workload (height field + spheres):
    primary, one diffuse bounce, shadow rays; the eight swept layouts and the
    quantised bvh2 layouts."""
    sc = scenes.config2_scene(side=181, n_spheres=64)
    tris = sc.triangles()
    prim = scenes.config2_primary(320, 180)
    ob = oracle_mod.BVH2(tris)
    h = ob.closest(prim)
    bounce = scenes.bounce_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"], seed=21)
    shadow = scenes.shadow_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"])
    eb = ob.closest(bounce)
    es = ob.any(shadow)
    for name, d in sc_mod.sweep_layouts(extended=True).items():
        bvh = sc_mod.scion_build(sc.verts, d, sc.indices)
        assert_same_hits(gpu_closest(sc_mod, bvh, prim), h, name + " primary")
        assert_same_hits(gpu_closest(sc_mod, bvh, bounce), eb, name + " bounce")
        assert np.array_equal(gpu_any(sc_mod, bvh, shadow), es), name + " shadow"


def test_random_soup_incoherent(sc_mod, oracle_mod):
    rng = scenes.rng_for(31)
    n = 1 << 17
    verts = scenes.random_soup(rng, n, mu=math.log(0.002 * math.sqrt((1 << 23) / n)))
    tris = verts.reshape(-1, 9)
    rays = scenes.random_rays(rng, 1 << 15, (0, 0, 0), (1, 1, 1))
    short = rays.copy()
    short[:, 7] = 0.05
    ob = oracle_mod.BVH2(tris)
    exp = ob.closest(rays)
    eocc = ob.any(short)
    for name, d in sc_mod.sweep_layouts(extended=True, orders=True).items():
        bvh = sc_mod.scion_build(verts, d)
        for p in (None, dict(rays_per_fetch=1), dict(rays_per_fetch=1, ordered_children=2, threads_per_block=128),
                  dict(ordered_children=3), dict(rays_per_fetch=1, ordered_children=3), dict(rays_per_fetch=8),
                  dict(rays_per_fetch=16, threads_per_block=64), dict(rays_per_fetch=32),
                  # shallow shared stacks: the ring kernels (own-box, 2/4-wide) spill and refill
                  # constantly; 5 and 12 round down to 4 and 8 there
                  dict(smem_stack=1), dict(smem_stack=5, rays_per_fetch=1), dict(smem_stack=12, ordered_children=3),
                  # stack entries in registers, spilling into shallow or default shared parts
                  dict(reg_stack=2), dict(reg_stack=4, rays_per_fetch=4), dict(reg_stack=4, smem_stack=1),
                  dict(reg_stack=2, smem_stack=5, rays_per_fetch=1, ordered_children=3)):
            assert_same_hits(gpu_closest(sc_mod, bvh, rays, params=p), exp, name + " " + str(p))
            assert np.array_equal(gpu_any(sc_mod, bvh, short, params=p), eocc), name + " " + str(p)


def test_concurrent_streams_same_bvh_and_host_tracer(sc_mod, oracle_mod):
    """Traces of one BVH issued on several streams at once (each stream has its
    own work counter) and the pipelined host-buffer tracer give the oracle's
    results."""
    rng = scenes.rng_for(41)
    verts = scenes.random_soup(rng, 1 << 16, mu=np.log(0.01))
    tris = verts.reshape(-1, 9)
    rays = scenes.random_rays(rng, 200_000, (0, 0, 0), (1, 1, 1))
    short = rays.copy()
    short[:, 7] = 0.05
    ob = oracle_mod.BVH2(tris)
    exp, eocc = ob.closest(rays), ob.any(short)
    bvh = sc_mod.scion_build(verts, sc_mod.layout(width=4, box_layout="soa", prim_ref="direct"))
    d = torch.from_numpy(rays).cuda()
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = [torch.empty((rays.shape[0], 4), dtype=torch.int32, device="cuda") for _ in streams]
    for _ in range(3):
        for st, o in zip(streams, outs):
            o.fill_(0)
            st.wait_stream(torch.cuda.current_stream())
            sc_mod.scion_trace_closest(bvh, d, o, stream=st)
        torch.cuda.synchronize()
        for o in outs:
            assert_same_hits(sc_mod.split_hits(o), exp, "concurrent")
    h_r = torch.from_numpy(rays).pin_memory()
    h_s = torch.from_numpy(short).pin_memory()
    h_o = torch.empty((rays.shape[0], 4), dtype=torch.int32).pin_memory()
    h_a = torch.empty((rays.shape[0],), dtype=torch.int32).pin_memory()
    h_o2 = torch.empty((rays.shape[0], 4), dtype=torch.int32).pin_memory()
    tracer = sc_mod.HostTracer(n_streams=3, chunk_rays=30_000)
    for p, phases in ((None, None), (dict(rays_per_fetch=1), None), (None, [[0], [1, 2]]),
                      (dict(rays_per_fetch=8), [[2], [0], [1]])):
        h_o.fill_(0)
        h_o2.fill_(0)
        h_a.fill_(7)
        tracer.trace([(bvh, h_r, h_o, "closest", p), (bvh, h_s, h_a, "any", p), (bvh, h_r, h_o2, "closest", p)],
                     phases)
        torch.cuda.synchronize()
        assert_same_hits(sc_mod.split_hits(h_o), exp, f"host tracer {p} {phases}")
        assert_same_hits(sc_mod.split_hits(h_o2), exp, f"host tracer {p} {phases}")
        assert np.array_equal(h_a.numpy().astype(np.uint32), eocc)
    # no staging copies: the kernels read rays from and write results to the
    # pinned host buffers in place, phases ordered by events
    direct = sc_mod.HostTracer(n_streams=2, zero_copy=True)
    for phases in (None, [[1], [0, 2]]):
        h_o.fill_(0)
        h_o2.fill_(0)
        h_a.fill_(7)
        direct.trace([(bvh, h_r, h_o, "closest", None), (bvh, h_s, h_a, "any", None),
                      (bvh, h_r, h_o2, "closest", dict(rays_per_fetch=8))], phases)
        torch.cuda.synchronize()
        assert_same_hits(sc_mod.split_hits(h_o), exp, f"in place {phases}")
        assert_same_hits(sc_mod.split_hits(h_o2), exp, f"in place {phases}")
        assert np.array_equal(h_a.numpy().astype(np.uint32), eocc)
    got = sc_mod.scion_trace_closest(bvh, h_r)  # pinned in, pinned out
    torch.cuda.synchronize()
    assert not got.is_cuda and got.is_pinned()
    assert_same_hits(sc_mod.split_hits(got), exp, "pinned host buffers")
    # pageable host memory cannot be reached from a kernel: rejected before any launch
    L = sc_mod.lib()
    pageable = np.ascontiguousarray(rays[:64])
    d_out = torch.empty((64, 4), dtype=torch.int32, device="cuda")
    st = L.scion_trace_closest(bvh.handle, ctypes.c_void_p(pageable.ctypes.data), 64,
                               ctypes.c_void_p(d_out.data_ptr()), None, None)
    assert st == 1
    st = L.scion_trace_any(bvh.handle, ctypes.c_void_p(d.data_ptr()), 64,
                           ctypes.c_void_p(np.zeros(64, np.int32).ctypes.data), None, None)
    assert st == 1
    # a growing chunk size (7,000 rays first, doubling up to 30,000)
    ramp = sc_mod.HostTracer(n_streams=2, chunk_rays=30_000, first_chunk_rays=7_000)
    h_o.fill_(0)
    h_a.fill_(7)
    ramp.trace([(bvh, h_r, h_o, "closest", None), (bvh, h_s, h_a, "any", None)], [[0], [1]])
    torch.cuda.synchronize()
    assert_same_hits(sc_mod.split_hits(h_o), exp, "host tracer, growing chunks")
    assert np.array_equal(h_a.numpy().astype(np.uint32), eocc)
    assert sc_mod.scion_get_status(bvh) == 0


def test_bvh_from_another_device_is_rejected(sc_mod):
    """Every call that takes a BVH checks that it lives on the current device:
    a BVH recorded as another GPU's is rejected with INVALID_ARG before
    anything is issued, and works again once its own device is restored."""
    L = sc_mod.lib()
    L.scion_debug_set_bvh_device.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.scion_debug_set_bvh_device.restype = ctypes.c_int
    sc = scenes.config1_scene()
    bvh = sc_mod.scion_build(sc.verts, sc_mod.layout(width=4, box_layout="soa"), sc.indices)
    rays = torch.from_numpy(scenes.config1_rays()[:256]).cuda()
    pts = torch.tensor([[0.1, 0.2, 0.5, float("inf")]], device="cuda")
    dv = torch.from_numpy(sc.verts).cuda()
    dev = torch.cuda.current_device()
    expected = sc_mod.scion_trace_closest(bvh, rays).clone()
    assert L.scion_debug_set_bvh_device(bvh.handle, dev + 1) == 0
    try:
        calls = (lambda: sc_mod.scion_trace_closest(bvh, rays), lambda: sc_mod.scion_trace_any(bvh, rays),
                 lambda: sc_mod.scion_query_closest_point(bvh, pts), lambda: sc_mod.scion_refit(bvh, dv))
        for call in calls:
            with pytest.raises(sc_mod.ScionError) as e:
                call()
            assert e.value.status == 1 and "built on device" in str(e.value), str(e.value)
    finally:
        assert L.scion_debug_set_bvh_device(bvh.handle, dev) == 0
    got = sc_mod.scion_trace_closest(bvh, rays)
    torch.cuda.synchronize()
    assert torch.equal(got, expected)
