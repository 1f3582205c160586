"""Batching (config 4, scaled down): many scenes of uneven size, each with its
own ray batch and an autotuned layout, traced in one persistent launch (also
captured in a CUDA graph and replayed). Hits must be bit-identical to
per-scene launches and to the CPU oracle."""
import numpy as np
import pytest

from paper_2511_15028_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15028_gb300 import build as b
    b.build()
    from paper_2511_15028_gb300 import autotune, scion
    scion.lib()
    return scion, autotune


@pytest.fixture(scope="module")
def workload(mods):
    scion, autotune = mods
    wl = scenes.config4_workload(n_scenes=24, scale=0.02)
    tuner = autotune.Autotuner(prim_refs=("direct", "indirect"), sample=2048, reps=1)
    chosen, rays = [], []
    for i, (sc, r) in enumerate(wl):
        d = torch.from_numpy(r).cuda()
        chosen.append(tuner.tune(i, sc.verts, sc.indices, d))
        rays.append(d)
    return wl, chosen, rays


def test_batched_equals_plain_and_oracle(mods, workload, oracle_mod):
    scion, _ = mods
    wl, chosen, rays = workload
    bvhs = [c.bvh for c in chosen]
    params = [c.params for c in chosen]
    batch = scion.Batch(bvhs, rays, params=params)
    assert batch.info()["batched_scenes"] == len(wl) and batch.info()["plain_scenes"] == 0
    hits = batch.launch()
    torch.cuda.synchronize()
    for i, (sc, r) in enumerate(wl):
        plain = scion.scion_trace_closest(bvhs[i], rays[i], params=params[i])
        torch.cuda.synchronize()
        assert torch.equal(hits[i], plain), i
        if sc.n_tris * r.shape[0] <= 4e8:
            exp = oracle_mod.closest_brute(sc.triangles(), r)
        else:
            exp = oracle_mod.BVH2(sc.triangles()).closest(r)
        got = scion.split_hits(hits[i])
        assert got.tobytes() == exp.tobytes(), i
        assert scion.scion_get_status(bvhs[i]) == 0
    # relaunching the same batch gives the same hits (self-resetting counters)
    before = [h.clone() for h in hits]
    for h in hits:
        h.fill_(0)
    batch.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(before, hits))


def test_batched_cuda_graph_replay(mods, workload):
    scion, _ = mods
    wl, chosen, rays = workload
    batch = scion.Batch([c.bvh for c in chosen], rays, params=[c.params for c in chosen])
    batch.launch()
    torch.cuda.synchronize()
    ref = [h.clone() for h in batch.hits]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.launch(stream=s)
    for _ in range(3):
        for h in batch.hits:
            h.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(ref, batch.hits))


def test_batched_mixed_layouts_fall_back_per_scene(mods, oracle_mod):
    """Layouts outside the batched families (indirect children, BVH2 SoA)
    still give correct hits, through their own launches."""
    scion, _ = mods
    wl = scenes.config4_workload(seed=77, n_scenes=6, scale=0.01)
    descs = [scion.layout(width=4, child_ref="indirect"), scion.layout(box_layout="soa"),
             scion.layout(width=8, box_prec="u8"), scion.layout(width=4, box_layout="soa"),
             scion.layout(width=2, box_prec="f16"), scion.layout(width=8, box_prec="f16", box_layout="soa")]
    bvhs, rays = [], []
    for (sc, r), d in zip(wl, descs):
        bvhs.append(scion.scion_build(sc.verts, d, sc.indices))
        rays.append(torch.from_numpy(r).cuda())
    batch = scion.Batch(bvhs, rays)
    info = batch.info()
    assert info["batched_scenes"] == 3 and info["plain_scenes"] == 3
    hits = batch.launch()
    torch.cuda.synchronize()
    for i, (sc, r) in enumerate(wl):
        exp = oracle_mod.BVH2(sc.triangles()).closest(r)
        assert scion.split_hits(hits[i]).tobytes() == exp.tobytes(), i


def test_batched_rejects_camera_ray_tiles(mods):
    """raster_width is a plain-launch parameter: a batch asked for it fails
    at creation, before any launch."""
    scion, _ = mods
    wl = scenes.config4_workload(seed=78, n_scenes=2, scale=0.01)
    bvhs = [scion.scion_build(sc.verts, scion.layout(width=4, box_layout="soa"), sc.indices) for sc, _ in wl]
    rays = [torch.from_numpy(r).cuda() for _, r in wl]
    with pytest.raises(scion.ScionError) as e:
        scion.Batch(bvhs, rays, params=[dict(raster_width=64), {}])
    assert e.value.status == 1


def test_config4_full_size(mods, oracle_mod):
    """The full batching workload: 64 scenes of 1K-2M triangles with 1K-1M
    rays each, layouts and parameters picked by the autotuner as the
    benchmark does, in one launch captured in a CUDA graph. Every hit equals
    the per-scene plain launch's, and 4,096 sampled rays per scene (all rays
    of smaller batches) equal the oracle's (brute force where cheap, else its
    BVH2)."""
    scion, autotune = mods
    wl = scenes.config4_workload(seed=1004)
    assert len(wl) == 64
    tuner = autotune.Autotuner()
    chosen, rays = [], []
    for i, (sc, r) in enumerate(wl):
        d = torch.from_numpy(r).cuda()
        chosen.append(tuner.tune(i, sc.verts, sc.indices, d))
        rays.append(d)
    bvhs = [c.bvh for c in chosen]
    params = [c.params for c in chosen]
    batch = scion.Batch(bvhs, rays, params=params)
    assert batch.info()["plain_scenes"] == 0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.launch(stream=s)
    for h in batch.hits:
        h.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(1404)
    for i, (sc, r) in enumerate(wl):
        plain = scion.scion_trace_closest(bvhs[i], rays[i], params=params[i])
        torch.cuda.synchronize()
        assert torch.equal(batch.hits[i], plain), f"scene {i}: batched != plain"
        pick = np.arange(r.shape[0]) if r.shape[0] <= 4096 else np.sort(rng.choice(r.shape[0], 4096, replace=False))
        tris = sc.triangles()
        if sc.n_tris * pick.size <= 4e8:
            exp = oracle_mod.closest_brute(tris, r[pick])
        else:
            exp = oracle_mod.BVH2(tris).closest(r[pick])
        got = scion.split_hits(batch.hits[i])[pick]
        assert got.tobytes() == exp.tobytes(), f"scene {i} ({sc.name}, {chosen[i].name}) vs oracle"
        assert scion.scion_get_status(bvhs[i]) == 0


def test_batched_every_family_and_fetch_mode(mods, oracle_mod):
    """Every node family of the batched kernel, with direct and indirect
    triangles, under warp batches and warp refill at several thresholds and
    child orders, in one launch: hits equal the oracle's."""
    scion, _ = mods
    fams = [dict(), dict(box_prec="q16"), dict(width=4, box_layout="soa"), dict(width=4, box_layout="soa", box_prec="f16"),
            dict(width=4, box_layout="soa", box_prec="u8", order="bfs"), dict(width=8, box_layout="soa", box_prec="f16"),
            dict(width=8, box_prec="u8"), dict(width=8, box_layout="soa", box_prec="u8", order="treelet")]
    modes = [{}, dict(rays_per_fetch=1), dict(rays_per_fetch=8, ordered_children=2),
             dict(rays_per_fetch=31, ordered_children=3), dict(ordered_children=2)]
    wl = scenes.config4_workload(seed=79, n_scenes=16, scale=0.01)
    bvhs, rays, params = [], [], []
    for i, (sc, r) in enumerate(wl):
        kw = dict(fams[i % len(fams)], prim_ref="direct" if i < 8 else "indirect")
        bvhs.append(scion.scion_build(sc.verts, scion.layout(**kw), sc.indices))
        rays.append(torch.from_numpy(r).cuda())
        params.append(modes[i % len(modes)])
    batch = scion.Batch(bvhs, rays, params=params)
    assert batch.info() == {"batched_scenes": 16, "plain_scenes": 0}
    for _ in range(2):  # the counters reset themselves between launches
        for h in batch.hits:
            h.fill_(-1)
        hits = batch.launch()
        torch.cuda.synchronize()
        for i, (sc, r) in enumerate(wl):
            exp = oracle_mod.BVH2(sc.triangles()).closest(r)
            assert scion.split_hits(hits[i]).tobytes() == exp.tobytes(), (i, params[i])
            assert scion.scion_get_status(bvhs[i]) == 0
    with pytest.raises(scion.ScionError):  # register stack tiers are for plain launches
        scion.Batch(bvhs[:1], rays[:1], params=[dict(reg_stack=4)])
