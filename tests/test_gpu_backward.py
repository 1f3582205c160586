"""Differentiation (config 5): L = sum w t + a u + b v on the config-1 scene
and rays. The GPU backward (FP32 atomic scatter) is checked against the FP64
CPU reference gradient and against central differences, and the autograd
wrapper returns the same numbers."""
import ctypes

import numpy as np
import pytest

from paper_2511_15028_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15028_gb300 import build as b
    b.build()
    from paper_2511_15028_gb300 import scion
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    tris = sc.triangles()
    w, a, bb = scenes.config5_weights(rays.shape[0])
    g = np.stack([w, a, bb], -1).astype(np.float32)
    hits = oracle_mod.closest_brute(tris, rays)
    gv64, gr64 = oracle_mod.grad(tris, sc.indices, sc.verts.shape[0], rays, hits, g)
    return scion, sc, rays, tris, g, hits, gv64, gr64


def _abs_scale(sc, rays, hits, g, tris):
    """Per-vertex sum of |contribution| (FP64), the scale of the FP32
    summation error."""
    hit = hits["prim"] != 0xFFFFFFFF
    p = tris[hits["prim"][hit]].astype(np.float64).reshape(-1, 3, 3)
    d = rays[hit, 4:7].astype(np.float64)
    c1 = -(p[:, 1] - p[:, 0])
    c2 = -(p[:, 2] - p[:, 0])
    x12, x20, x01 = np.cross(c1, c2), np.cross(c2, d), np.cross(d, c1)
    det = np.sum(d * x12, axis=1)
    gg = g[hit].astype(np.float64)
    lam = (gg[:, :1] * x12 + gg[:, 1:2] * x20 + gg[:, 2:3] * x01) / det[:, None]
    u = hits["u"][hit].astype(np.float64)
    v = hits["v"][hit].astype(np.float64)
    wts = np.stack([1 - u - v, u, v], -1)
    S = np.zeros((sc.verts.shape[0], 3))
    ids = sc.indices[hits["prim"][hit]]
    for j in range(3):
        np.add.at(S, ids[:, j], np.abs(wts[:, j:j + 1] * lam))
    return S


@pytest.mark.parametrize("layout", ["bvh2_aos_f32_indirect", "bvh8_aos_u8_direct", "bvh4_soa_f32_direct"])
def test_backward_matches_fp64_reference(setup, layout):
    scion, sc, rays, tris, g, hits, gv64, gr64 = setup
    bvh = scion.scion_build(sc.verts, scion.sweep_layouts()[layout], sc.indices)
    d_rays = torch.from_numpy(rays).cuda()
    h = scion.scion_trace_closest(bvh, d_rays)
    assert scion.split_hits(h).tobytes() == hits.tobytes()
    gv, gr = scion.scion_trace_backward(bvh, d_rays, h, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    gv = gv.cpu().numpy().astype(np.float64)
    gr = gr.cpu().numpy().astype(np.float64)
    S = _abs_scale(sc, rays, hits, g, tris)
    assert np.all(np.abs(gv - gv64) <= 1e-5 * S + 1e-6)
    ray_ref = np.zeros_like(gr)
    ray_ref[:, 0:3] = gr64[:, 0:3]
    ray_ref[:, 4:7] = gr64[:, 3:6]
    assert np.all(np.abs(gr - ray_ref) <= 1e-6 * np.abs(ray_ref) + 1e-6)
    assert np.all(gr[:, 3] == 0) and np.all(gr[:, 7] == 0)
    miss = hits["prim"] == 0xFFFFFFFF
    assert np.all(gr[miss] == 0)


def test_backward_against_central_differences(setup, oracle_mod):
    scion, sc, rays, tris, g, hits, gv64, gr64 = setup
    fv, fr = oracle_mod.grad_fd(tris, sc.indices, sc.verts.shape[0], rays, hits, g, 1e-4)
    bvh = scion.scion_build(sc.verts, scion.layout(), sc.indices)
    d_rays = torch.from_numpy(rays).cuda()
    h = scion.scion_trace_closest(bvh, d_rays)
    gv, _ = scion.scion_trace_backward(bvh, d_rays, h, torch.from_numpy(g).cuda())
    gv = gv.cpu().numpy().astype(np.float64)
    assert np.abs(gv - fv).max() <= 1e-4 * np.abs(fv).max()


def test_autograd_function_and_accumulation(setup):
    scion, sc, rays, tris, g, hits, gv64, gr64 = setup
    bvh = scion.scion_build(sc.verts, scion.layout(width=8, box_prec="u8"), sc.indices)
    verts = torch.from_numpy(sc.verts).cuda().requires_grad_(True)
    r = torch.from_numpy(rays).cuda().requires_grad_(True)
    t, u, v, prim = scion.trace_fn().apply(verts, r, bvh)
    hit = prim != -1
    w = torch.from_numpy(g).cuda()
    loss = (torch.where(hit, t, torch.zeros_like(t)) * w[:, 0]).sum() + (u * w[:, 1]).sum() + (v * w[:, 2]).sum()
    loss.backward()
    S = _abs_scale(sc, rays, hits, g, tris)
    gvv = verts.grad.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gvv - gv64) <= 1e-5 * S + 1e-6)
    # accumulation: a second backward adds the same amount again
    gv2, _ = scion.scion_trace_backward(bvh, r.detach(), scion.scion_trace_closest(bvh, r.detach()),
                                        torch.from_numpy(g).cuda(), grad_verts=verts.grad.clone(),
                                        want_ray_grads=False)
    assert np.all(np.abs(gv2.cpu().numpy() - 2 * gvv) <= 2e-5 * S + 2e-6)


def test_backward_and_counters_take_device_buffers_only(setup):
    """Gradients and visit counters are added with device atomics: host
    buffers are rejected before any launch."""
    scion = setup[0]
    sc = scenes.config1_scene()
    bvh = scion.scion_build(sc.verts, scion.layout(), sc.indices)
    rays = torch.from_numpy(scenes.config1_rays()[:64]).cuda()
    hits = scion.scion_trace_closest(bvh, rays)
    L = scion.lib()
    host_grad = np.zeros((sc.verts.shape[0], 3), np.float32)
    g_tuv = torch.zeros((64, 3), device="cuda")
    st = L.scion_trace_backward(bvh.handle, ctypes.c_void_p(rays.data_ptr()), ctypes.c_void_p(hits.data_ptr()),
                                ctypes.c_void_p(g_tuv.data_ptr()), 64, ctypes.c_void_p(host_grad.ctypes.data),
                                None, None)
    assert st == 1
    out = torch.empty((64, 4), dtype=torch.int32, device="cuda")
    host_cnt = np.zeros(4, np.uint64)
    st = L.scion_trace_stats(bvh.handle, ctypes.c_void_p(rays.data_ptr()), 64, 0, ctypes.c_void_p(out.data_ptr()),
                             None, None, ctypes.c_void_p(host_cnt.ctypes.data))
    assert st == 1
