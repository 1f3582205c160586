"""Host-side packer checks (no GPU): every layout of one logical tree decodes
back to the same leaves, every decoded box encloses its subtree (quantised
bounds always enclose the original, Section 9.1 footnote; round-trip
soundness, App. B), node sizes match Table 1 where the layouts coincide, and
invalid descriptors are rejected."""
import itertools
import math

import numpy as np
import pytest

from paper_2511_15028_gb300 import scenes, scion


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2511_15028_gb300 import build as b
    b.build()
    scion.lib()


def all_layouts():
    out = []
    for w, lay, prec, cref, pref, order in itertools.product(
            (2, 4, 8), ("aos", "soa"), ("f32", "f16", "u8"), ("direct", "indirect"),
            ("direct", "indirect"), ("dfs", "bfs", "treelet")):
        own = w == 2 and prec == "f32"
        if own and cref == "direct" and order != "dfs":
            continue
        out.append(dict(width=w, box_layout=lay, box_prec=prec, child_ref=cref, prim_ref=pref, order=order))
    return out


def walk(dec):
    """Triangle ids under every node; checks each node is reached once."""
    info = dec.info
    n = info["n_nodes"]
    if n == 0:
        return {}, []
    own = info["own_box"] == 1
    seen = np.zeros(n, np.int32)
    order = []
    stack = [0]
    while stack:
        x = stack.pop()
        seen[x] += 1
        order.append(x)
        for k in range(8):
            if dec.kind[x, k] == 1:
                assert 0 <= dec.a[x, k] < n
                stack.append(int(dec.a[x, k]))
    assert np.all(seen == 1), "every node reached exactly once from the root"
    sub = {}
    leaves = []
    for x in reversed(order):
        ids = []
        for k in range(8):
            if dec.kind[x, k] == 1:
                ids.append(sub[int(dec.a[x, k])])
            elif dec.kind[x, k] == 2:
                f, c = int(dec.a[x, k]), int(dec.c[x, k])
                assert 1 <= c <= 16
                lid = dec.leaf_ids[f:f + c]
                leaves.append(tuple(sorted(lid.tolist())))
                ids.append(lid)
        sub[x] = np.concatenate(ids) if ids else np.zeros(0, np.uint32)
    return sub, leaves


def check_enclosure(dec, sub, tris):
    own = dec.info["own_box"] == 1
    P = tris.reshape(-1, 3, 3)
    for x, ids in sub.items():
        if own:
            lo, hi = dec.own_boxes[x, :3], dec.own_boxes[x, 3:]
            q = P[ids].reshape(-1, 3)
            assert np.all(q >= lo) and np.all(q <= hi)
        else:
            for k in range(8):
                kd = dec.kind[x, k]
                if kd == 0:
                    continue
                if kd == 1:
                    cid = sub[int(dec.a[x, k])]
                else:
                    f, c = int(dec.a[x, k]), int(dec.c[x, k])
                    cid = dec.leaf_ids[f:f + c]
                q = P[cid].reshape(-1, 3)
                lo, hi = dec.boxes[x, k, :3], dec.boxes[x, k, 3:]
                assert np.all(q >= lo) and np.all(q <= hi), (x, k)


@pytest.mark.parametrize("kw", all_layouts(), ids=lambda kw: "-".join(str(v) for v in kw.values()))
def test_roundtrip_config1_all_layouts(kw):
    sc = scenes.config1_scene()
    tris = sc.triangles()
    dec = scion.scion_debug_build_host(sc.verts, scion.layout(**kw), sc.indices)
    sub, leaves = walk(dec)
    ids = np.sort(np.concatenate([np.array(l) for l in leaves]))
    assert np.array_equal(ids, np.arange(4096)), "leaf entries hold every triangle exactly once"
    check_enclosure(dec, sub, tris)
    # the logical BVH2 is shared by every layout: same leaves everywhere
    ref = scion.scion_debug_build_host(sc.verts, scion.layout(), sc.indices)
    _, ref_leaves = walk(ref)
    assert sorted(leaves) == sorted(ref_leaves)
    assert dec.info["n_leaf_entries"] == 4096


def test_pbrt_node_size_and_wide_sizes():
    sc = scenes.config1_scene()
    d = scion.scion_debug_build_host(sc.verts, scion.layout(), sc.indices).info
    assert d["node_stride"] == 32 and d["node_bytes"] == 32 * d["n_nodes"]  # Table 1: pbrt 32 B
    soa = scion.scion_debug_build_host(sc.verts, scion.layout(box_layout="soa"), sc.indices).info
    assert soa["node_bytes"] == 32 * soa["n_nodes"]  # pbrt-soaos: still 32 B per node
    expect = {(4, "f32", "direct"): 128, (8, "f16", "direct"): 128, (8, "u8", "direct"): 96,
              (8, "u8", "indirect"): 96, (8, "f32", "direct"): 224, (4, "u8", "direct"): 64,
              (2, "f16", "direct"): 32}
    for (w, p, c), size in expect.items():
        i = scion.scion_debug_build_host(sc.verts, scion.layout(width=w, box_prec=p, child_ref=c), sc.indices).info
        assert i["node_stride"] == size, (w, p, c)


def test_soup_extreme_coordinates_enclosure():
    """Boxes stay enclosing for tiny, huge and offset coordinates (u8 frames
    with extreme exponents, f16 overflow to infinity)."""
    rng = scenes.rng_for(12)
    for scale, offset in ((1e-30, 0.0), (1e-3, 1e4), (1e30, 0.0), (1.0, -3e5), (1e5, 1e5)):
        v = scenes.random_soup(rng, 3000, mu=math.log(0.01)) * scale + offset
        v = v.astype(np.float32)
        tris = v.reshape(-1, 9)
        for prec in ("f32", "f16", "u8"):
            for w in (2, 4, 8):
                dec = scion.scion_debug_build_host(v, scion.layout(width=w, box_prec=prec))
                sub, leaves = walk(dec)
                check_enclosure(dec, sub, tris)
                assert sum(len(l) for l in leaves) == 3000


def test_degenerate_scenes():
    # a flat scene (zero extent in z), a single triangle, all triangles at one point
    sc = scenes.config1_scene()
    flat = sc.verts.copy()
    flat[:, 2] = 0.5
    for prec in ("f32", "f16", "u8"):
        dec = scion.scion_debug_build_host(flat, scion.layout(width=8, box_prec=prec), sc.indices)
        sub, _ = walk(dec)
        check_enclosure(dec, sub, flat[sc.indices].reshape(-1, 9))
    one = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    for kw in ({}, dict(width=8, box_prec="u8"), dict(width=4, box_prec="f16", child_ref="indirect")):
        dec = scion.scion_debug_build_host(one, scion.layout(**kw))
        sub, leaves = walk(dec)
        assert leaves == [(0,)]
        check_enclosure(dec, sub, one.reshape(1, 9))
    pt = np.zeros((30, 3), np.float32) + np.float32(0.25)
    dec = scion.scion_debug_build_host(pt, scion.layout(width=8, box_prec="u8", leaf_max=2))
    _, leaves = walk(dec)
    assert sum(len(l) for l in leaves) == 10 and max(len(l) for l in leaves) <= 2


def test_nonfinite_triangles_left_out_and_empty_scene():
    v = scenes.config1_scene().triangles().reshape(-1, 3).copy()
    v[5] = np.nan
    v[100] = np.inf
    dec = scion.scion_debug_build_host(v, scion.layout(width=4))
    _, leaves = walk(dec)
    ids = sorted(i for l in leaves for i in l)
    assert 1 not in ids and 33 not in ids and len(ids) == 4094
    empty = scion.scion_debug_build_host(np.zeros((0, 3), np.float32), scion.layout())
    assert empty.info["n_nodes"] == 0 and empty.info["n_leaf_entries"] == 0
    allbad = np.full((9, 3), np.nan, np.float32)
    assert scion.scion_debug_build_host(allbad, scion.layout(width=8)).info["n_nodes"] == 0


def test_invalid_descriptors_rejected():
    v = scenes.config1_scene().triangles().reshape(-1, 3)
    bad = [dict(width=3), dict(width=16), dict(box_prec=3), dict(order=3), dict(leaf_max=17),
           dict(sah_bins=1), dict(sah_bins=65), dict(reserved=1),
           dict(width=2, box_prec=0, child_ref=0, order=1), dict(width=2, box_prec=0, child_ref=0, order=2)]
    for b in bad:
        d = scion.layout()
        for k, val in b.items():
            setattr(d, k, val)
        with pytest.raises(scion.ScionError) as e:
            scion.scion_debug_build_host(v, d)
        assert e.value.status in (1, 2)
    # soup with a vertex count that is not 3 * n, indices out of range
    with pytest.raises(scion.ScionError):
        scion.scion_debug_build_host(v[:10], scion.layout(), None)
    with pytest.raises(scion.ScionError):
        scion.scion_debug_build_host(v, scion.layout(), np.array([[0, 1, 10 ** 6]], np.uint32))


def test_orders_keep_siblings_contiguous_for_indirect_refs():
    sc = scenes.config2_scene(side=65, n_spheres=16)
    for order in ("dfs", "bfs", "treelet"):
        dec = scion.scion_debug_build_host(sc.verts, scion.layout(width=4, child_ref="indirect", order=order),
                                           sc.indices)
        for x in range(dec.info["n_nodes"]):
            kids = [int(dec.a[x, k]) for k in range(8) if dec.kind[x, k] == 1]
            assert kids == list(range(kids[0], kids[0] + len(kids))) if kids else True
    # BFS: node index grows with depth
    dec = scion.scion_debug_build_host(sc.verts, scion.layout(width=4, order="bfs"), sc.indices)
    depth = np.zeros(dec.info["n_nodes"], int)
    for x in range(dec.info["n_nodes"]):
        for k in range(8):
            if dec.kind[x, k] == 1:
                depth[dec.a[x, k]] = depth[x] + 1
    assert np.all(np.diff(depth) >= 0)
    # DFS direct: the pbrt own-box layout puts the left child right after its parent
    dec = scion.scion_debug_build_host(sc.verts, scion.layout(), sc.indices)
    for x in range(dec.info["n_nodes"]):
        if dec.kind[x, 0] == 1:
            assert dec.a[x, 0] == x + 1


def _f16_bits_to_float(h):
    return float(np.array([h], np.uint16).view(np.float16)[0])


def test_f16_directed_rounding_against_numpy():
    """round_down(x) is the largest binary16 <= x and round_up(x) the
    smallest >= x, checked against numpy's float16 (round to nearest)."""
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-9, 6, 2000),
                         [0.0, -0.0, 1.0, -1.0, 65504.0, -65504.0, 65519.0, 70000.0, -70000.0,
                          6e-8, -6e-8, 1e-9, 2.0 ** -24, 2.0 ** -14, 1e30, -1e30]]).astype(np.float32)
    for x in xs:
        x = float(x)
        lo = _f16_bits_to_float(scion.scion_debug_f16_round(x, -1))
        hi = _f16_bits_to_float(scion.scion_debug_f16_round(x, +1))
        assert lo <= x <= hi
        assert scion.scion_debug_f16_decode(scion.scion_debug_f16_round(x, -1)) == lo
        with np.errstate(over="ignore"):
            rn = float(np.float16(x))
        assert rn in (lo, hi) or (math.isinf(rn) and abs(x) < 65520)
        if lo != hi:
            # adjacent binary16 values: nothing representable strictly between
            a = np.array([lo], np.float16).view(np.uint16)[0]
            nxt = np.nextafter(np.float16(lo), np.float16(np.inf)) if math.isfinite(lo) else None
            if nxt is not None and math.isfinite(hi):
                assert float(nxt) == hi, (x, lo, hi, a)
