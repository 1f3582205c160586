"""Host-side packer checks (no GPU): every layout of one logical tree decodes
back to the same leaves, every decoded box encloses its subtree (quantised
bounds always enclose the original, Section 9.1 footnote; round-trip
soundness, App. B), node sizes match Table 1 where the layouts coincide, and
invalid descriptors are rejected."""
import math
from fractions import Fraction

import numpy as np
import pytest

from layout_cases import OWN_ONLY, WORLD_GRID, all_layouts
from paper_2511_15028_gb300 import scenes, scion


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2511_15028_gb300 import build as b
    b.build()
    scion.lib()


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
              (2, "f16", "direct"): 32, (8, "u16", "direct"): 160, (4, "u16", "indirect"): 96}
    for (w, p, c), size in expect.items():
        i = scion.scion_debug_build_host(sc.verts, scion.layout(width=w, box_prec=p, child_ref=c), sc.indices).info
        assert i["node_stride"] == size, (w, p, c)
    # Table 1 bvh2 codecs: sg-pbrt-q16 16 B (also -soaos: 12 + 4), sg-eq 12 B,
    # sg-eq-align16 16 B, pbrt-soaos-align16 32 + 8 B
    for kw, per_node in ((dict(box_prec="q16"), 16), (dict(box_prec="q16", box_layout="soa"), 16),
                         (dict(box_prec="eq10"), 12), (dict(box_prec="eq10", align=16), 16),
                         (dict(box_prec="q16", box_layout="soa", align=16), 20),
                         (dict(box_layout="soa", align=16), 40), (dict(align=16), 32),
                         (dict(box_prec="slab"), 16)):
        i = scion.scion_debug_build_host(sc.verts, scion.layout(**kw), sc.indices).info
        assert i["own_box"] == 1 and i["node_bytes"] == per_node * i["n_nodes"], kw


def test_soup_extreme_coordinates_enclosure():
    """Boxes stay enclosing for tiny, huge and offset coordinates (u8 frames
    with extreme exponents, f16 overflow to infinity)."""
    rng = scenes.rng_for(12)
    for scale, offset in ((1e-30, 0.0), (1e-3, 1e4), (1e30, 0.0), (1.0, -3e5), (1e5, 1e5)):
        v = scenes.random_soup(rng, 3000, mu=math.log(0.01)) * scale + offset
        v = v.astype(np.float32)
        tris = v.reshape(-1, 9)
        for prec in ("f32", "f16", "u8", "u16") + OWN_ONLY:
            for w in ((2,) if prec in OWN_ONLY else (2, 4, 8)):
                dec = scion.scion_debug_build_host(v, scion.layout(width=w, box_prec=prec))
                sub, leaves = walk(dec)
                check_enclosure(dec, sub, tris)
                assert sum(len(l) for l in leaves) == 3000
                if prec in WORLD_GRID:
                    check_world_grid(dec)


def test_degenerate_scenes():
    # a flat scene (zero extent in z), a single triangle, all triangles at one point
    sc = scenes.config1_scene()
    flat = sc.verts.copy()
    flat[:, 2] = 0.5
    for w, prec in ((8, "f32"), (8, "f16"), (8, "u8"), (2, "q16"), (2, "eq10")):
        dec = scion.scion_debug_build_host(flat, scion.layout(width=w, box_prec=prec), sc.indices)
        sub, _ = walk(dec)
        check_enclosure(dec, sub, flat[sc.indices].reshape(-1, 9))
        if prec in WORLD_GRID:
            check_world_grid(dec)
    one = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    for kw in ({}, dict(width=8, box_prec="u8"), dict(width=4, box_prec="f16", child_ref="indirect"),
               dict(box_prec="q16"), dict(box_prec="eq10")):
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
    bad = [dict(width=3), dict(width=16), dict(box_prec=7), dict(order=3), dict(leaf_max=17),
           dict(sah_bins=1), dict(sah_bins=65), dict(align=1), dict(align=32),
           dict(width=4, box_prec=3), dict(width=8, box_prec=4), dict(box_prec=3, leaf_max=16),
           dict(box_prec=4, box_layout=1), dict(width=2, box_prec=3, child_ref=0, order=1),
           dict(width=4, box_prec=6), dict(box_prec=6, box_layout=1), dict(box_prec=6, child_ref=0, order=2),
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


# ------------------------------------------------------------ world-grid codecs
def _f32_round(fr, mode):
    """Exact rounding of a rational to binary32: 'rn' (ties to even), 'rd'
    (toward -inf) or 'ru' (toward +inf)."""
    x = np.float32(float(fr))
    cands = [np.nextafter(x, np.float32(-np.inf)), x, np.nextafter(x, np.float32(np.inf))]
    cands = [c for c in cands if np.isfinite(c)]
    if mode == "rd":
        return max((c for c in cands if Fraction(float(c)) <= fr), key=float)
    if mode == "ru":
        return min((c for c in cands if Fraction(float(c)) >= fr), key=float)
    best = min(abs(Fraction(float(c)) - fr) for c in cands)
    near = [c for c in cands if abs(Fraction(float(c)) - fr) == best]
    return near[0] if len(near) == 1 else [c for c in near if int(np.array(c).view(np.uint32)) % 2 == 0][0]


def _world_grid_codes(dec):
    """(lo codes [n,3], hi codes [n,3], words [n]) read from the raw bytes."""
    d = dec.info
    n, stride = d["n_nodes"], d["node_stride"]
    raw = dec.nodes.reshape(n, stride)
    if d["node2_bytes"]:  # q16 -soaos: code records + a word array
        codes = raw[:, :12].copy().view("<u2").reshape(n, 6).astype(np.int64)
        return codes[:, :3], codes[:, 3:], dec.nodes2.view("<u4").copy()
    if stride == 16 and dec.frame[6] == 0.0:  # q16 AoS: 6 codes + word
        codes = raw[:, :12].copy().view("<u2").reshape(n, 6).astype(np.int64)
        return codes[:, :3], codes[:, 3:], raw[:, 12:16].copy().view("<u4").ravel()
    w = raw[:, :12].copy().view("<u4").reshape(n, 3)  # eq10: lo word, hi word, node word
    unpack = lambda x: np.stack([(x >> 20) & 1023, (x >> 10) & 1023, x & 1023], 1).astype(np.int64)  # noqa: E731
    return unpack(w[:, 0]), unpack(w[:, 1]), w[:, 2]


def check_world_grid(dec, limit=None):
    """Decode every node's box from its codes with exact rational arithmetic
    (q16: coordinate = RN(code * step + wlo); eq10, the App. D.1 grid with
    one outward rounding: lo = RD(code * bin + wlo), hi = RU(whi - code * bin))
    and compare
    with the packer's decode bit for bit; the node word's count and child
    fields must match the decoded tree."""
    n = dec.info["n_nodes"]
    if n == 0:
        return
    lo_c, hi_c, words = _world_grid_codes(dec)
    f = [Fraction(float(x)) for x in dec.frame]
    eq = dec.frame[6] != 0.0  # eq10 bins are never 0; q16 leaves these slots 0
    idx = range(n) if limit is None else np.random.default_rng(0).choice(n, min(n, limit), replace=False)
    for x in idx:
        for a in range(3):
            if eq:
                lo = _f32_round(f[a] + lo_c[x, a] * f[6 + a], "rd")
                hi = _f32_round(f[3 + a] - hi_c[x, a] * f[6 + a], "ru")
                assert 0 <= lo_c[x, a] <= 1023 and 0 <= hi_c[x, a] <= 1023
            else:
                lo = _f32_round(lo_c[x, a] * f[3 + a] + f[a], "rn")
                hi = _f32_round(hi_c[x, a] * f[3 + a] + f[a], "rn")
            got_lo, got_hi = dec.own_boxes[x, a], dec.own_boxes[x, 3 + a]
            assert np.array([lo], np.float32).view(np.uint32)[0] == np.array([got_lo], np.float32).view(np.uint32)[0]
            assert np.array([hi], np.float32).view(np.uint32)[0] == np.array([got_hi], np.float32).view(np.uint32)[0]
        w = int(words[x])
        cnt = w & 15
        if cnt:
            assert dec.kind[x, 0] == 2 and dec.c[x, 0] == cnt and dec.a[x, 0] == w >> 4
        else:
            assert dec.kind[x, 0] == 1 and dec.kind[x, 1] == 1 and (w >> 4) & 3 <= 2


@pytest.mark.parametrize("kw", [dict(box_prec="q16"), dict(box_prec="q16", box_layout="soa"),
                                dict(box_prec="q16", box_layout="soa", align=16),
                                dict(box_prec="eq10"), dict(box_prec="eq10", align=16),
                                dict(box_prec="q16", child_ref="indirect", order="bfs")],
                         ids=lambda kw: "-".join(str(v) for v in kw.values()))
def test_world_grid_codecs_decode_independently(kw):
    sc = scenes.config1_scene()
    dec = scion.scion_debug_build_host(sc.verts, scion.layout(**kw), sc.indices)
    check_world_grid(dec)
    sub, _ = walk(dec)
    check_enclosure(dec, sub, sc.triangles())


def test_world_grid_frames_and_slack():
    """The grid spans the root box; eq10's bins follow App. D.1
    (bins_inv = RD(1023 / RU(whi - wlo)), bin = RD(1 / bins_inv)); q16's step is
    the smallest float with RN(65535 * step + wlo) >= whi. Every decoded box
    is at most about one grid step (plus the build pad) looser than its
    subtree's bounds."""
    sc = scenes.config2_scene(side=65, n_spheres=16)
    tris = sc.triangles()
    P = tris.reshape(-1, 3, 3)
    for prec in WORLD_GRID:
        dec = scion.scion_debug_build_host(sc.verts, scion.layout(box_prec=prec), sc.indices)
        sub, _ = walk(dec)
        fr = dec.frame
        root_lo, root_hi = dec.own_boxes[0, :3], dec.own_boxes[0, 3:]
        for a in range(3):
            wlo = Fraction(float(fr[a]))
            if prec == "eq10":
                whi = Fraction(float(fr[3 + a]))
                L = _f32_round(whi - wlo, "ru")
                L = L if L > 0 else np.float32(1.0)
                inv = _f32_round(Fraction(1023) / Fraction(float(L)), "rd")
                assert fr[6 + a] == _f32_round(1 / Fraction(float(inv)), "rd")
                step = float(fr[6 + a])
                assert root_lo[a] <= fr[a] and root_hi[a] >= fr[3 + a]
            else:
                step = float(fr[3 + a])
                top = _f32_round(65535 * Fraction(step) + wlo, "rn")
                below = _f32_round(65535 * Fraction(float(np.nextafter(np.float32(step), np.float32(0)))) + wlo, "rn")
                assert root_lo[a] == fr[a] and top >= root_hi[a] and below < root_hi[a]
        for x, ids in sub.items():
            q = P[ids].reshape(-1, 3)
            tlo, thi = q.min(0).astype(np.float64), q.max(0).astype(np.float64)
            ext = float(np.max(thi - tlo))
            mag = float(np.max(np.abs(np.concatenate([tlo, thi]))))
            pad = 2.0 ** -19 * (ext + mag) + 1e-30
            steps = fr[6:9] if prec == "eq10" else fr[3:6]
            assert np.all(tlo - dec.own_boxes[x, :3] <= 2 * steps + pad), (prec, x)
            assert np.all(dec.own_boxes[x, 3:] - thi <= 2 * steps + pad), (prec, x)


def test_world_grid_limits():
    """leaf_max above the 4-bit count field and layouts outside the codec's
    forms are rejected; a scene of one point builds (zero-extent grid)."""
    pt = np.zeros((30, 3), np.float32) + np.float32(-7.5)
    for prec in WORLD_GRID:
        dec = scion.scion_debug_build_host(pt, scion.layout(box_prec=prec, leaf_max=15))
        _, leaves = walk(dec)
        assert sum(len(l) for l in leaves) == 10
        check_world_grid(dec)


def test_shared_slab_carried_boxes_independent():
    """Shared-slab layout (Section 8.3): decode the carried boxes top-down from
    the raw node bytes (root = frame; a child takes its parent's box with one
    plane replaced), compare with the library's decode, and check that every
    carried box encloses its subtree's triangles and lies inside its parent's."""
    sc = scenes.config2_scene(side=65, n_spheres=16)
    tris = sc.triangles()
    for kw in (dict(box_prec="slab"), dict(box_prec="slab", child_ref="indirect", order="bfs")):
        dec = scion.scion_debug_build_host(sc.verts, scion.layout(**kw), sc.indices)
        n = dec.info["n_nodes"]
        raw = dec.nodes.reshape(n, 16)
        planes = raw[:, :8].copy().view("<f4")
        field = raw[:, 8:12].copy().view("<u4").ravel()
        meta = raw[:, 12:16].copy().view("<u4").ravel()
        box = np.full((n, 6), np.nan, np.float32)
        box[0] = dec.frame[:6]
        for x in range(n):  # parents precede children in every order
            if meta[x] & 0xFFFF:
                continue
            ax = (meta[x] >> 16) & 3
            l, r = (x + 1, x + field[x]) if kw.get("child_ref") != "indirect" else (field[x], field[x] + 1)
            box[l] = box[x]
            box[r] = box[x]
            box[l, 3 + ax] = planes[x, 0]
            box[r, ax] = planes[x, 1]
            assert box[l, 3 + ax] <= box[x, 3 + ax] and box[r, ax] >= box[x, ax]
        assert np.array_equal(box.view(np.uint32), dec.own_boxes.view(np.uint32))
        sub, _ = walk(dec)
        check_enclosure(dec, sub, tris)
