"""Every layout descriptor the test suite sweeps (CPU packer tests and GPU
parity tests use the same list)."""
import itertools

WORLD_GRID = ("q16", "eq10")


def all_layouts():
    out = []
    for w, lay, prec, cref, pref, order in itertools.product(
            (2, 4, 8), ("aos", "soa"), ("f32", "f16", "u8", "u16") + WORLD_GRID, ("direct", "indirect"),
            ("direct", "indirect"), ("dfs", "bfs", "treelet")):
        if prec in WORLD_GRID and (w != 2 or (prec == "eq10" and lay == "soa")):
            continue
        own = w == 2 and prec in ("f32",) + WORLD_GRID
        if own and cref == "direct" and order != "dfs":
            continue
        out.append(dict(width=w, box_layout=lay, box_prec=prec, child_ref=cref, prim_ref=pref, order=order))
    # the -align16 variants of Table 1 that change the record size
    for prec, lay in (("eq10", "aos"), ("q16", "soa"), ("f32", "soa")):
        for cref in ("direct", "indirect"):
            out.append(dict(width=2, box_layout=lay, box_prec=prec, child_ref=cref, prim_ref="indirect",
                            order="dfs", align=16))
    return out
