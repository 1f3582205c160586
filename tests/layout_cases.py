"""Every layout descriptor the test suite sweeps (CPU packer tests and GPU
parity tests use the same list)."""
import itertools

WORLD_GRID = ("q16", "eq10")
OWN_ONLY = WORLD_GRID + ("slab",)  # width-2 own-box-like nodes only


def all_layouts():
    out = []
    for w, lay, prec, cref, pref, order in itertools.product(
            (2, 4, 8), ("aos", "soa"), ("f32", "f16", "u8", "u16") + OWN_ONLY, ("direct", "indirect"),
            ("direct", "indirect"), ("dfs", "bfs", "treelet")):
        if prec in OWN_ONLY and (w != 2 or (prec in ("eq10", "slab") and lay == "soa")):
            continue
        own = w == 2 and prec in ("f32",) + OWN_ONLY
        if own and cref == "direct" and order != "dfs":
            continue
        out.append(dict(width=w, box_layout=lay, box_prec=prec, child_ref=cref, prim_ref=pref, order=order))
    # the -align16 variants of Table 1 that change the record size
    for prec, lay in (("eq10", "aos"), ("q16", "soa"), ("f32", "soa")):
        for cref in ("direct", "indirect"):
            out.append(dict(width=2, box_layout=lay, box_prec=prec, child_ref=cref, prim_ref="indirect",
                            order="dfs", align=16))
    return out
