"""scion_trace_closest_noalloc: the closest-hit entry point for callers that
cannot allocate device memory while tracing (an application whose arena owns
all device memory, or a latency-bound thread that must stay out of the
driver's allocator).

Called through the C ABI; its hits must equal scion_trace_closest's on two
calls in a row (both share the library's static scratch array). Kept in a file
of its own that pytest collects last."""
import ctypes

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
    L = scion.lib()
    P = ctypes.c_void_p
    L.scion_trace_closest_noalloc.argtypes = [P, P, ctypes.c_uint64, P, ctypes.POINTER(scion.TraceParams), P]
    L.scion_trace_closest_noalloc.restype = ctypes.c_int
    return scion


def _noalloc(scion, bvh, rays, hits, stream):
    return scion.lib().scion_trace_closest_noalloc(
        bvh.handle, ctypes.c_void_p(rays.data_ptr()), rays.shape[0], ctypes.c_void_p(hits.data_ptr()),
        None, ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_plain_entry_point_twice(sc_mod):
    scion = sc_mod
    stream = torch.cuda.current_stream()
    cases = [(scenes.config1_scene(), scenes.config1_rays())]
    rng = scenes.rng_for(77)
    soup = scenes.Scene(scenes.random_soup(rng, 1 << 14, mu=np.log(0.02)), None)
    cases.append((soup, scenes.random_rays(rng, 50_000, (0, 0, 0), (1, 1, 1))))
    # the first call on a device does the one-time set-up (looks up the static
    # array's device address, which may load the library's device module)
    sc0, r0 = cases[0]
    b0 = scion.scion_build(sc0.verts, scion.layout(), sc0.indices)
    r0 = torch.from_numpy(r0[:64]).cuda()
    h0 = torch.empty((64, 4), dtype=torch.int32, device="cuda")
    assert _noalloc(scion, b0, r0, h0, stream) == 0
    torch.cuda.synchronize()
    for sc, rays_np in cases:
        rays = torch.from_numpy(rays_np).cuda()
        for name, desc in scion.sweep_layouts().items():
            bvh = scion.scion_build(sc.verts, desc, sc.indices)
            ref = scion.scion_trace_closest(bvh, rays)
            out = [torch.full_like(ref, -1), torch.full_like(ref, -1)]
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            for o in out:  # two calls in a row share the static scratch
                assert _noalloc(scion, bvh, rays, o, stream) == 0
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, "the call allocated device memory"
            for o in out:
                # the tolerance of every parity test here: bit-exact
                assert torch.equal(o, ref), name
            assert scion.scion_get_status(bvh) == 0


def test_noalloc_rejects_oversize_and_bad_arguments(sc_mod):
    scion = sc_mod
    sc = scenes.config1_scene()
    bvh = scion.scion_build(sc.verts, scion.layout(), sc.indices)
    rays = torch.from_numpy(scenes.config1_rays()).cuda()
    hits = torch.empty((rays.shape[0], 4), dtype=torch.int32, device="cuda")
    L = scion.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.scion_trace_closest_noalloc(bvh.handle, ctypes.c_void_p(rays.data_ptr()), 1 << 62,
                                       ctypes.c_void_p(hits.data_ptr()), None, s)
    assert st == 1 and "2^62" in scion.last_error()
    assert L.scion_trace_closest_noalloc(None, None, 5, None, None, s) == 1
    assert L.scion_trace_closest_noalloc(bvh.handle, ctypes.c_void_p(rays.data_ptr()), 0, None, None, s) == 0
    # camera-ray tiles: same hits as 32 consecutive rays; refilled warps cannot take tiles
    ref = scion.scion_trace_closest(bvh, rays)
    tiles = scion.TraceParams(raster_width=128)
    st = L.scion_trace_closest_noalloc(bvh.handle, ctypes.c_void_p(rays.data_ptr()), rays.shape[0],
                                       ctypes.c_void_p(hits.data_ptr()), ctypes.byref(tiles), s)
    torch.cuda.synchronize()
    assert st == 0 and torch.equal(hits, ref)
    # pinned host rays and hits are read and written in place; pageable host
    # memory is rejected before anything is issued
    h_rays = rays.cpu().pin_memory()
    h_hits = torch.full((rays.shape[0], 4), -1, dtype=torch.int32).pin_memory()
    st = L.scion_trace_closest_noalloc(bvh.handle, ctypes.c_void_p(h_rays.data_ptr()), rays.shape[0],
                                       ctypes.c_void_p(h_hits.data_ptr()), None, s)
    torch.cuda.synchronize()
    assert st == 0 and torch.equal(h_hits, ref.cpu())
    pageable = np.zeros((64, 4), np.int32)
    assert L.scion_trace_closest_noalloc(bvh.handle, ctypes.c_void_p(rays.data_ptr()), 64,
                                         ctypes.c_void_p(pageable.ctypes.data), None, s) == 1
    bad = scion.TraceParams(raster_width=128, rays_per_fetch=4)
    assert L.scion_trace_closest_noalloc(bvh.handle, ctypes.c_void_p(rays.data_ptr()), rays.shape[0],
                                         ctypes.c_void_p(hits.data_ptr()), ctypes.byref(bad), s) == 1
