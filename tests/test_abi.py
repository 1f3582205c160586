"""The C-ABI library builds, loads without a GPU, exports every function the
public headers declare, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in os.listdir(INCLUDE):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(scion_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libscion():
    from paper_2511_15028_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for n in ("scion_build", "scion_trace_closest", "scion_trace_any", "scion_bvh_info",
              "scion_get_status", "scion_destroy", "scion_status_string", "scion_trace_stats"):
        assert n in names


def test_every_declared_symbol_is_exported(libscion):
    missing = [n for n in declared_functions() if not hasattr(libscion, n)]
    assert not missing, missing


def test_status_strings_and_argument_errors_without_gpu(libscion):
    libscion.scion_status_string.restype = ctypes.c_char_p
    for s in range(8):
        assert libscion.scion_status_string(s)
    # null handles / outputs are rejected synchronously, no device touched
    libscion.scion_bvh_info.argtypes = [ctypes.c_void_p] * 5
    assert libscion.scion_bvh_info(None, None, None, None, None) == 1
    libscion.scion_trace_closest.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert libscion.scion_trace_closest(None, None, 5, None, None, None) == 1
    libscion.scion_build.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p(1)
    assert libscion.scion_build(None, 3, None, 1, None, None, ctypes.byref(out)) == 1
    assert out.value is None
    libscion.scion_destroy.argtypes = [ctypes.c_void_p]
    libscion.scion_destroy(None)


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle and the library links nothing of it."""
    pkg = os.path.join(ROOT, "paper_2511_15028_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "oracle.h" not in text, f


def test_python_binding_rejects_unreachable_buffers_without_gpu():
    """Ray and result tensors must live on the GPU or in pinned host memory (the
    kernels read pinned host memory in place); anything else, or the wrong dtype
    or a strided view, is a TypeError before the library is called."""
    torch = pytest.importorskip("torch")
    from paper_2511_15028_gb300 import scion
    pageable = torch.zeros(4, 8)
    assert not pageable.is_pinned()
    cases = [(scion.scion_trace_closest, pageable), (scion.scion_trace_any, pageable),
             (scion.scion_query_closest_point, torch.zeros(4, 4)), (scion.scion_trace_stats, pageable),
             (scion.scion_trace_closest, torch.zeros(4, 8, dtype=torch.float64)),
             (scion.scion_trace_closest, torch.zeros(8, 4).t())]
    for fn, t in cases:
        with pytest.raises(TypeError):
            fn(None, t)


def test_camera_ray_tiles_cover_every_ray_once(libscion):
    """Host logic of raster_width: the slot count the kernels loop over
    (scion_debug_raster_slots) ends at the last 8x4 tile holding a ray, and the
    kernels' slot -> pixel mapping (slot s: tile s // 32, lane s % 32 at column
    8 (t mod tiles_x) + lane mod 8, row 4 (t div tiles_x) + lane div 8) reaches
    every ray exactly once, for ragged widths and partial last rows."""
    libscion.scion_debug_raster_slots.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
    libscion.scion_debug_raster_slots.restype = ctypes.c_uint64
    for n in list(range(1, 40)) + [100, 127, 128, 129, 1000, 4096]:
        assert libscion.scion_debug_raster_slots(n, 0) == n
        for w in (1, 2, 3, 7, 8, 9, 16, 17, 33, 100, 128, 1 << 20):
            slots = libscion.scion_debug_raster_slots(n, w)
            tiles_x = (w + 7) // 8
            # the last tile holding a ray, from the rays' side
            last = max((i // w // 4) * tiles_x + (i % w) // 8 for i in range(n))
            assert slots == 32 * (last + 1), (n, w, slots)
            s = np.arange(slots)
            t, lane = s // 32, s % 32
            px = (t % tiles_x) * 8 + (lane & 7)
            py = (t // tiles_x) * 4 + (lane >> 3)
            rid = py * w + px
            hit = rid[(px < w) & (rid < n)]
            assert np.array_equal(np.sort(hit), np.arange(n)), (n, w)
    # widths next to 2^32, where a 32-bit tile count would wrap to zero: every
    # ray lies in the first tile row
    for w in (2**31 + 1, 2**32 - 8, 2**32 - 7, 2**32 - 1):
        for n in (1, 8, 9, 100):
            assert libscion.scion_debug_raster_slots(n, w) == 32 * ((n - 1) // 8 + 1), (n, w)
