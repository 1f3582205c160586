#!/usr/bin/env python
"""Benchmark: closest-hit / any-hit traversal throughput per layout.

Workload (one step): the coherent + incoherent scene of 1,373,138 triangles
(724 x 724 fBm height field + 256 icospheres), 1920 x 1080 primary camera rays
(closest hit), one cosine-weighted diffuse bounce ray per primary hit (closest
hit) and one shadow ray per primary hit toward a point light (any hit), all
inputs resident in HBM. Every swept layout is timed (the eight layouts of
the four node families with direct and indirect triangles, and the quantised
bvh2 layouts sg-pbrt-q16, -soaos, sg-eq and sg-eq-align16); the headline
value is the best layout's whole-step Mrays/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun every rank traces its own copy
of the workload (weak scaling) and the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "closest-hit Mrays/s & BVH MB per layout; % BW roofline; batched/bwd vs plain"
WORKLOAD = ("coherent+incoherent: fBm 724x724 height field + 256 icospheres (1,373,138 tris); "
            "1920x1080 primary (closest) + 1 diffuse bounce per hit (closest) + 1 shadow per hit (any)")
L2_FLUSH_BYTES = 512 << 20


def trimmed_mean(xs):
    """Paper's protocol (Section 9.1): of 9 runs drop the 2 lowest and 2
    highest and average the rest; for other counts trim 2/9 on each side."""
    xs = sorted(xs)
    k = int(round(len(xs) * 2 / 9)) if len(xs) >= 5 else 0
    core = xs[k:len(xs) - k] if len(xs) > 2 * k else xs
    return float(sum(core) / len(core))


# ------------------------------------------------------------------ algorithmic bytes
def node_load_bytes(desc) -> int:
    """Bytes one node visit loads (128-bit loads of the used part of a node)."""
    w, prec, cref = desc.width, desc.box_prec, desc.child_ref
    if w == 2 and prec == 0:
        return 32
    if prec == 3:  # q16 own-box node: 12 B of codes + 4 B word
        return 16
    if prec == 4:  # eq10 own-box node: 12 B (16 B aligned)
        return 16 if desc.align == 16 else 12
    if prec == 6:  # shared-slab node: planes + field + meta
        return 16
    elem = {0: 4, 1: 2, 2: 1, 5: 2}[prec]
    used = (16 if prec in (2, 5) else 0) + w * 6 * elem + (4 * w if cref == 0 else 8 + w)
    return (used + 15) // 16 * 16


def tri_load_bytes(desc, indexed: bool) -> int:
    if desc.prim_ref == 0:
        return 48
    return 4 + (12 if indexed else 0) + 48


# ------------------------------------------------------------------ profiled traffic
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "trace_kernel_traffic.txt")
KERNEL_SOURCES = ("trace.cuh", "trace_inst.cu", "layout.h", "kernels.h")


def _strip_comments(src: str) -> str:
    """C/C++ source without comments and with whitespace collapsed: edits of
    comments or layout leave the hash (and so the recorded counters) valid."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_sources_hash() -> str:
    """Hash of the traversal kernel's code (comments stripped) and of the
    nvcc flags it is built with."""
    import hashlib

    from paper_2511_15028_gb300 import build as native_build
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(_strip_comments(open(os.path.join(ROOT, "paper_2511_15028_gb300", "csrc", f)).read()).encode())
    h.update(" ".join(native_build.ARCH + native_build.NVCC_FLAGS[:-1]).encode())
    return h.hexdigest()


def profiled_traffic(workload: str, layout: str, query: str):
    """(DRAM bytes, L2 bytes) per launch of the traversal kernel on this
    workload, layout and query, from the committed ncu summary
    profiles/trace_kernel_traffic.txt; None when it holds no such capture or
    the kernel's code has changed since it was taken."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    sha, rows = None, {}
    for line in open(TRAFFIC_FILE):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "kernel_sources_sha256":
            sha = f[1]
        elif len(f) >= 4 and f[0] in ("coherent", "incoherent"):
            kv = dict(x.split("=", 1) for x in f[3:] if "=" in x)
            rows[(f[0], f[1], f[2])] = kv
    if sha is None or sha != kernel_sources_hash():
        return None
    kv = rows.get((workload, layout, query))
    if kv is None:
        return None
    return {"dram_bytes": int(kv["dram_bytes"]), "l2_bytes": int(kv["l2_bytes"]),
            "fetch": kv.get("fetch"), "source": os.path.relpath(TRAFFIC_FILE, ROOT)}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampled every 10 ms while the benchmark runs; only samples
    taken inside the timed windows (host wall-clock) are kept."""
    FIELDS = ("timestamp,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = bus_id
        self.proc = None
        self.windows = []
        self.path = os.path.join("/tmp", f"scion_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except OSError:
            self.proc = None

    def window(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            if self.bus_id and self.bus_id.lower()[-12:] not in f[1].lower():
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            if any(a - 0.005 <= ts <= b + 0.005 for a, b in self.windows):
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        num = lambda x: float(x) if x.replace(".", "", 1).isdigit() else None  # noqa: E731
        sm = [v for v in (num(r[2]) for r in rows) if v is not None]
        mx = [v for v in (num(r[3]) for r in rows) if v is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ L2 read peak
def measure_l2_peak(scion, torch, sizes_mib=(16, 32, 48, 64), target_ms=1.0, trials=7):
    """L2 read bandwidth of this GPU, measured live: the library's read probe
    (16-byte loads that bypass L1, every SM) streams an L2-resident buffer many
    times in one launch, timed with CUDA events; best of `trials` launches per
    buffer size. The roofline peak is the largest rate over the sizes."""
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = {}
    for mib in sizes_mib:
        buf = torch.randint(0, 1 << 30, ((mib << 20) // 4,), dtype=torch.int32, device="cuda")
        nbytes = buf.numel() * 4
        scion.scion_debug_read_bandwidth(buf, 1, sink)  # bring it into L2
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        scion.scion_debug_read_bandwidth(buf, 8, sink)
        b.record()
        b.synchronize()
        reps = max(8, int(8 * target_ms / max(a.elapsed_time(b), 1e-3)))
        best = 0.0
        for _ in range(trials):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            scion.scion_debug_read_bandwidth(buf, reps, sink)
            b.record()
            b.synchronize()
            best = max(best, nbytes * reps / (a.elapsed_time(b) / 1e3) / 1e9)
        out[f"{mib}MiB"] = round(best, 1)
        del buf
    return {"peak_gbs": max(out.values()), "by_size_gbs": out,
            "how": "ld.global.cg 16-byte loads over an L2-resident buffer, every SM, one launch of many passes, "
                   f"best of {trials} launches per size (CUDA events)"}


# ------------------------------------------------------------------ workload
def make_workload(scion, torch, dev, primary_desc):
    from paper_2511_15028_gb300 import scenes
    sc = scenes.config2_scene()
    prim = scenes.config2_primary()
    bvh = scion.scion_build(sc.verts, primary_desc, sc.indices)
    d_prim = torch.from_numpy(prim).to(dev)
    h = scion.split_hits(scion.scion_trace_closest(bvh, d_prim))
    bounce = scenes.bounce_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"], seed=2002)
    shadow = scenes.shadow_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"])
    return sc, prim, bounce, shadow


def flush_l2(buf):
    buf.zero_()


# Traversal parameters tried per layout and kind of ray (fetch mode x child
# order); any-hit ignores the child order.
_BASE_MODES = {"warp_batch": {}, "refill1": {"rays_per_fetch": 1}, "refill4": {"rays_per_fetch": 4},
               "refill8": {"rays_per_fetch": 8}, "refill16": {"rays_per_fetch": 16},
               "warp_batch/nearest_first": {"ordered_children": 3},
               "refill1/nearest_first": {"rays_per_fetch": 1, "ordered_children": 3},
               "refill8/nearest_first": {"rays_per_fetch": 8, "ordered_children": 3}}
# each mode also with the newest 4 stack entries in registers (and 2 for the
# two most used modes)
FETCH_MODES = dict(_BASE_MODES)
FETCH_MODES.update({f"{k}/reg4": {**v, "reg_stack": 4} for k, v in _BASE_MODES.items()})
FETCH_MODES.update({f"{k}/reg2": {**_BASE_MODES[k], "reg_stack": 2} for k in ("warp_batch", "refill8")})
# Primary rays are a row-major 1920-wide image: warps can take 8x4 pixel tiles.
PRIMARY_RASTER = 1920
RASTER_MODES = {"tiles": {"raster_width": PRIMARY_RASTER},
                "tiles/nearest_first": {"raster_width": PRIMARY_RASTER, "ordered_children": 3},
                "tiles/reg4": {"raster_width": PRIMARY_RASTER, "reg_stack": 4},
                "tiles/nearest_first/reg4": {"raster_width": PRIMARY_RASTER, "ordered_children": 3,
                                             "reg_stack": 4}}


def mode_params(name):
    return (FETCH_MODES[name] if name in FETCH_MODES else RASTER_MODES[name]) or None


def pick_fetch(scion, torch, bvh, fn, rays, out, reps=3, extra=None):
    """Traversal parameters chosen by measurement (the autotuner's choice for
    one layout and one kind of ray): the fastest candidate, and every
    candidate's best time in ms."""
    best, best_t, trials = None, None, {}
    cands = FETCH_MODES if fn is scion.scion_trace_closest else {
        k: v for k, v in FETCH_MODES.items() if "nearest" not in k}
    if extra:
        cands = {**cands, **extra}
    for name, p in cands.items():
        fn(bvh, rays, out, params=p or None)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn(bvh, rays, out, params=p or None)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        t = min(ts)
        trials[name] = round(t, 4)
        if best_t is None or t < best_t:
            best, best_t = name, t
    return best, trials


def time_layout(scion, torch, bvh, rays, outs, steps, warmup, flush_buf, sampler=None, fixed=None):
    """K timed steps of primary closest hit, then bounce closest hit and
    shadow any hit (both made from the primary hits, so they wait for it and
    run concurrently on two streams). Events on each launch's own stream
    around each launch; the step is timed on the main stream from before the
    primary launch to after both others have joined. Each kind of ray uses
    the fetch mode measured fastest for it."""
    d_p, d_b, d_s = rays
    o_p, o_b, o_s = outs
    fns = (scion.scion_trace_closest, scion.scion_trace_closest, scion.scion_trace_any)
    if fixed:  # modes given on the command line: no trials
        picks = [(m, {}) for m in fixed]
    else:
        picks = [pick_fetch(scion, torch, bvh, f, r, o, extra=RASTER_MODES if i == 0 else None)
                 for i, (f, r, o) in enumerate(zip(fns, rays, outs))]
    modes = [m for m, _ in picks]
    ps = [mode_params(m) for m in modes]
    stream = torch.cuda.current_stream()
    s_b, s_s = torch.cuda.Stream(), torch.cuda.Stream()

    def one_step(e=None):
        if e:
            e[0].record(stream)
        scion.scion_trace_closest(bvh, d_p, o_p, params=ps[0])
        if e:
            e[1].record(stream)
        s_b.wait_stream(stream)
        s_s.wait_stream(stream)
        if e:
            e[2].record(s_b)
        scion.scion_trace_closest(bvh, d_b, o_b, params=ps[1], stream=s_b)
        if e:
            e[3].record(s_b)
            e[4].record(s_s)
        scion.scion_trace_any(bvh, d_s, o_s, params=ps[2], stream=s_s)
        if e:
            e[5].record(s_s)
        stream.wait_stream(s_b)
        stream.wait_stream(s_s)
        if e:
            e[6].record(stream)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(steps)]
    t_start = time.time()
    for k in range(steps):
        flush_l2(flush_buf)
        one_step(ev[k])
    torch.cuda.synchronize()
    if sampler:
        sampler.window(t_start, time.time())
    per = np.array([[e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3]), e[4].elapsed_time(e[5])]
                    for e in ev])  # ms per launch
    step = np.array([e[0].elapsed_time(e[6]) for e in ev])
    return step, per, modes, [t for _, t in picks]


def e2e_layout(scion, torch, bvh, host_rays, steps, warmup, flush_buf, modes=("warp_batch",) * 3, zero_copy=True):
    """The same step through the public API from pinned host memory; bounce
    and shadow traces start after the primary traces. zero_copy: the kernels
    read each step's rays from, and write its results to, the pinned host
    buffers over the host link (no staging copies); otherwise every step
    copies its rays host->device and its results device->host, pipelined in
    chunks on three streams so that the copies overlap the traversal."""
    h_in = [torch.from_numpy(r).pin_memory() for r in host_rays]
    n = [r.shape[0] for r in host_rays]
    h_out = [torch.empty((n[0], 4), dtype=torch.int32).pin_memory(),
             torch.empty((n[1], 4), dtype=torch.int32).pin_memory(),
             torch.empty((n[2],), dtype=torch.int32).pin_memory()]
    ps = [mode_params(m) for m in modes]
    jobs = [(bvh, h_in[0], h_out[0], "closest", ps[0]), (bvh, h_in[1], h_out[1], "closest", ps[1]),
            (bvh, h_in[2], h_out[2], "any", ps[2])]
    tracer = scion.HostTracer(zero_copy=zero_copy)
    stream = torch.cuda.current_stream()
    phases = [[0], [1, 2]]  # bounce and shadow rays come from the primary hits
    for _ in range(warmup):
        tracer.trace(jobs, phases)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush_l2(flush_buf)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tracer.trace(jobs, phases)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    bi = sum(r.nbytes for r in host_rays)
    bo = sum(h.numel() * 4 for h in h_out)
    return times, bi, bo


# ------------------------------------------------------------------ CPU baseline (oracle)
def cpu_oracle_setup():
    """The CPU oracle's own copy of the workload: its BVH2 over the scene, the
    primary rays, and bounce / shadow rays generated from the oracle's own
    primary hits (nothing here comes from the GPU path)."""
    import oracle
    from paper_2511_15028_gb300 import scenes
    sc = scenes.config2_scene()
    prim = scenes.config2_primary()
    bvh = oracle.BVH2(sc.triangles(), bins=32, leaf_max=4)
    h = bvh.closest(prim)
    bounce = scenes.bounce_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"], seed=2002)
    shadow = scenes.shadow_rays(sc, prim, h["t"], h["u"], h["v"], h["prim"])
    return bvh, prim, bounce, shadow


def cpu_oracle_pass(bvh, prim, bounce, shadow):
    """One pass of the workload on the host cores; returns (seconds, rays)."""
    t0 = time.perf_counter()
    bvh.closest(prim)
    bvh.closest(bounce)
    bvh.any(shadow)
    return time.perf_counter() - t0, prim.shape[0] + bounce.shape[0] + shadow.shape[0]


def cpu_baseline(target_s: float = 12.0):
    import oracle
    bvh, prim, bounce, shadow = cpu_oracle_setup()
    secs, n = cpu_oracle_pass(bvh, prim, bounce, shadow)
    reps = max(1, min(200, int(math.ceil(target_s / max(secs, 1e-3)))))
    tot_s, tot_n = 0.0, 0
    for _ in range(reps):
        s_, n_ = cpu_oracle_pass(bvh, prim, bounce, shadow)
        tot_s += s_
        tot_n += n_
    return {"value": tot_n / tot_s / 1e6, "unit": "Mrays/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{reps} passes of the full step ({n} rays each: primary + bounce + shadow), "
                      f"oracle binned-SAH BVH2 traversal (build excluded), {tot_s:.1f} s total"}


def run_reference(args, rank):
    """The oracle as it stands, on the host cores, on the same workload: each
    step is one full pass (primary + bounce + shadow)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    bvh, prim, bounce, shadow = cpu_oracle_setup()
    times, counts = [], []
    for i in range(args.warmup + args.steps):
        secs, n = cpu_oracle_pass(bvh, prim, bounce, shadow)
        if i >= args.warmup:
            times.append(secs)
            counts.append(n)
    ms = trimmed_mean([t * 1e3 for t in times])
    val = float(np.mean(counts)) / (ms / 1e3) / 1e6
    thr = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mrays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "layout": "oracle BVH2 (32 bins, <=4 tris/leaf)"},
            "cpu_baseline": {"value": val, "unit": "Mrays/s", "cores": thr, "kind": "oracle",
                             "sample": "one full pass of the step per timed step"},
            "e2e": {"value": val, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ incoherent (config 3)
def pareto(points):
    """Names on the footprint-vs-throughput Pareto front (smaller MB, higher Mrays/s)."""
    front = []
    for n, (mb, mr) in points.items():
        if not any((mb2 <= mb and mr2 >= mr) and (mb2 < mb or mr2 > mr) for n2, (mb2, mr2) in points.items()):
            front.append(n)
    return sorted(front, key=lambda n: points[n][0])


def bench_incoherent(scion, torch, steps, warmup, hbm_peak, only=None, fixed=None):
    """2^23 random triangles and 2^23 random rays in the unit cube (BVH far
    larger than L2): closest hit (tmax inf) and any hit (tmax 0.05) for every
    swept layout, built from one logical BVH. fixed = (closest mode, any
    mode) skips the per-layout trials (to profile exactly those launches)."""
    from paper_2511_15028_gb300 import scenes
    t0 = time.time()
    sc = scenes.config3_scene()
    rays = torch.from_numpy(scenes.config3_rays()).cuda()
    short = rays.clone()
    short[:, 7] = 0.05
    gen_s = time.time() - t0
    lays = scion.sweep_layouts(extended=True, orders=True)
    if only:
        lays = {k: v for k, v in lays.items() if k in only}
    t0 = time.time()
    bvhs = scion.scion_build_many(sc.verts, list(lays.values()))
    build_s = time.time() - t0
    n = rays.shape[0]
    hits = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    occ = torch.empty((n,), dtype=torch.int32, device="cuda")
    out = {}
    for (name, desc), bvh in zip(lays.items(), bvhs):
        info = scion.scion_bvh_info(bvh)
        _, cc = scion.scion_trace_stats(bvh, rays, 0)
        _, ca = scion.scion_trace_stats(bvh, short, 1)
        cc, ca = cc.cpu().numpy(), ca.cpu().numpy()
        sn, st = node_load_bytes(desc), tri_load_bytes(desc, False)
        alg = {"closest": int(cc[3]) * 48 + int(cc[0]) * sn + int(cc[2]) * st,
               "any": int(ca[3]) * 36 + int(ca[0]) * sn + int(ca[2]) * st}
        res = {}
        for q, fn, r, o in (("closest", scion.scion_trace_closest, rays, hits),
                            ("any", scion.scion_trace_any, short, occ)):
            if fixed:
                mode, trials = fixed[0 if q == "closest" else 1], {}
            else:
                mode, trials = pick_fetch(scion, torch, bvh, fn, r, o, reps=2)
            p = FETCH_MODES[mode] or None
            for _ in range(warmup):
                fn(bvh, r, o, params=p)
            torch.cuda.synchronize()
            ts = []
            for _ in range(steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn(bvh, r, o, params=p)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            ms = trimmed_mean(ts)
            gbs = alg[q] / (ms / 1e3) / 1e9
            res[q] = {"ms": ms, "mrays_s": n / (ms / 1e3) / 1e6, "bytes_per_ray": alg[q] / n, "fetch_mode": mode,
                      "fetch_trials_ms": trials,
                      "alg_gbs": gbs, "roofline_frac_of_measured_hbm": gbs / hbm_peak}
        res["bvh_mb"] = (info["node_bytes"] + info["prim_bytes"]) / 1e6
        res["nodes_per_ray"] = {"closest": float(cc[0]) / n, "any": float(ca[0]) / n}
        res["tris_per_ray"] = {"closest": float(cc[2]) / n, "any": float(ca[2]) / n}
        out[name] = res
        scion.scion_destroy(bvh)
    best = max(out, key=lambda k: out[k]["closest"]["mrays_s"])
    best_any = max(out, key=lambda k: out[k]["any"]["mrays_s"])
    roof = {}
    for q, name in (("closest", best), ("any", best_any)):
        prof = profiled_traffic("incoherent", name, q)
        rq = out[name][q]
        roof[q] = {"bound": "hbm", "layout": name, "achieved": round(rq["alg_gbs"], 1), "peak": hbm_peak,
                   "unit": "GB/s", "frac": round(rq["roofline_frac_of_measured_hbm"], 4),
                   "traffic": prof["dram_bytes"] if prof else None,
                   "l2_traffic": prof["l2_bytes"] if prof else None,
                   "traffic_source": prof["source"] if prof else None,
                   "note": "the BVH is far larger than L2: the roof is the measured HBM copy bandwidth"}
    return {"tris": sc.n_tris, "rays": n, "gen_s": round(gen_s, 1), "build_layouts_s": round(build_s, 1),
            "roofline": roof, "layouts": out, "best_closest": best, "best_any": best_any,
            "pareto_closest": pareto({k: (v["bvh_mb"], v["closest"]["mrays_s"]) for k, v in out.items()}),
            "pareto_any": pareto({k: (v["bvh_mb"], v["any"]["mrays_s"]) for k, v in out.items()})}


def time_query(scion, torch, bvh, fn, rays, out, steps, warmup):
    """Trimmed-mean ms of one query in its measured-fastest traversal mode."""
    mode, trials = pick_fetch(scion, torch, bvh, fn, rays, out, reps=2)
    p = FETCH_MODES[mode] or None
    for _ in range(warmup):
        fn(bvh, rays, out, params=p)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn(bvh, rays, out, params=p)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return trimmed_mean(ts), mode


# ------------------------------------------------------------------ closest point query
def bench_cpq(scion, torch, steps, warmup, hbm_peak):
    """Closest point query (App. G): 2^20 points uniform in the coherent
    scene's box (the paper's query count), unbounded radius, on the swept
    layouts with direct triangles; throughput, visits and the algorithmic
    bytes fraction of the measured HBM bandwidth."""
    from paper_2511_15028_gb300 import scenes
    sc = scenes.config2_scene()
    rng = np.random.default_rng(2005)
    lo, hi = sc.verts.min(0) - 0.1, sc.verts.max(0) + 0.1
    n = 1 << 20
    pts = torch.from_numpy(np.concatenate([lo + (hi - lo) * rng.uniform(size=(n, 3)), np.full((n, 1), np.inf)],
                                          1).astype(np.float32)).cuda()
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    res = {}
    for name, desc in scion.sweep_layouts(extended=True).items():
        if name.endswith("indirect") or name.startswith("bvh2_slab"):  # slab: rays only
            continue
        bvh = scion.scion_build(sc.verts, desc, sc.indices)
        _, c = scion.scion_trace_stats(bvh, pts, 2)
        c = c.cpu().numpy()
        # an own-box visit reads its node and both children's nodes (the
        # children's boxes are bounded at the parent); a wide visit one node
        own = desc.width == 2 and desc.box_prec in (0, 3, 4)
        alg = (int(c[3]) * 32 + int(c[0]) * node_load_bytes(desc) * (3 if own else 1)
               + int(c[2]) * tri_load_bytes(desc, True))
        best, best_ms = None, None
        for mode, p in (("sorted", None), ("slot_order", {"ordered_children": 2})):
            scion.scion_query_closest_point(bvh, pts, out, params=p)
            torch.cuda.synchronize()
            ts = []
            for _ in range(warmup + steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                scion.scion_query_closest_point(bvh, pts, out, params=p)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            ms = trimmed_mean(ts[warmup:])
            if best_ms is None or ms < best_ms:
                best, best_ms = mode, ms
        info = scion.scion_bvh_info(bvh)
        res[name] = {"mpoints_s": n / (best_ms / 1e3) / 1e6, "ms": best_ms, "order": best,
                     "bvh_mb": (info["node_bytes"] + info["prim_bytes"]) / 1e6,
                     "nodes_per_point": float(c[0]) / n, "tris_per_point": float(c[2]) / n,
                     "alg_frac_of_measured_hbm": alg / (best_ms / 1e3) / 1e9 / hbm_peak}
        del bvh
    return {"points": n, "layouts": res,
            "pareto": pareto({k: (v["bvh_mb"], v["mpoints_s"]) for k, v in res.items()})}


# ------------------------------------------------------------------ GPU construction
def bench_build(scion, torch, steps, warmup):
    """Logical-BVH2 construction on the host (binned SAH, all host cores) and
    on the GPU (linear BVH), both packed by the same host packers; and the
    incoherent workload traced on both kinds of tree."""
    from paper_2511_15028_gb300 import scenes
    tiny = torch.tensor([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=torch.float32, device="cuda")
    scion.scion_build_gpu(tiny, scion.layout())  # first-call costs out of the timings
    out = {}
    sc2 = scenes.config2_scene()
    sc3 = scenes.config3_scene()
    for name, sc, ix in (("coherent_1373138_tris", sc2, sc2.indices), ("incoherent_8388608_tris", sc3, None)):
        dv = torch.from_numpy(sc.verts).cuda()
        dix = None if ix is None else torch.from_numpy(ix.astype(np.int32)).cuda()
        res = {"tris": sc.n_tris}
        lays = {"bvh4_soa_f32_direct": scion.layout(width=4, box_layout="soa", prim_ref="direct"),
                "bvh8_aos_u8_direct": scion.layout(width=8, box_prec="u8", prim_ref="direct")}
        trees = {}
        for builder in ("sah_host", "lbvh_gpu"):
            for lname, desc in lays.items():
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                bvh = (scion.scion_build(sc.verts, desc, ix) if builder == "sah_host"
                       else scion.scion_build_gpu(dv, desc, dix))
                wall = (time.perf_counter() - t0) * 1e3
                bt = scion.scion_bvh_build_times(bvh)
                info = scion.scion_bvh_info(bvh)
                res.setdefault(builder, {})[lname] = {
                    "logical_ms": round(bt["logical_ms"], 2), "pack_ms": round(bt["pack_ms"], 2),
                    "wall_ms": round(wall, 1), "n_nodes": info["n_nodes"], "depth": info["depth"],
                    "bvh_mb": (info["node_bytes"] + info["prim_bytes"]) / 1e6}
                trees[(builder, lname)] = bvh
        res["lbvh_logical_mtris_s"] = sc.n_tris / (res["lbvh_gpu"]["bvh4_soa_f32_direct"]["logical_ms"] / 1e3) / 1e6
        res["sah_logical_mtris_s"] = sc.n_tris / (res["sah_host"]["bvh4_soa_f32_direct"]["logical_ms"] / 1e3) / 1e6
        if sc is sc3:
            rays = torch.from_numpy(scenes.config3_rays()).cuda()
            short = rays.clone()
            short[:, 7] = 0.05
            n = rays.shape[0]
            hits = torch.empty((n, 4), dtype=torch.int32, device="cuda")
            occ = torch.empty((n,), dtype=torch.int32, device="cuda")
            tr = {}
            for (builder, lname), bvh in trees.items():
                mc, fc = time_query(scion, torch, bvh, scion.scion_trace_closest, rays, hits, steps, warmup)
                ma, fa = time_query(scion, torch, bvh, scion.scion_trace_any, short, occ, steps, warmup)
                tr[f"{builder}/{lname}"] = {"closest_mrays_s": n / (mc / 1e3) / 1e6, "closest_mode": fc,
                                            "any_mrays_s": n / (ma / 1e3) / 1e6, "any_mode": fa}
            # refit the SAH trees to a slightly moved soup (every vertex moves by
            # up to 1e-3, about half a triangle edge), then trace the moved scene
            moved = dv + 1e-3 * torch.sin(dv * 37.0 + torch.arange(3, device="cuda"))
            refit = {}
            for lname in lays:
                bvh = trees[("sah_host", lname)]
                scion.scion_refit(bvh, moved)  # first call allocates the scratch
                ts = []
                for k in range(steps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    scion.scion_refit(bvh, dv if k % 2 == 0 else moved)
                    b.record()
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                scion.scion_refit(bvh, moved)
                mc, fc = time_query(scion, torch, bvh, scion.scion_trace_closest, rays, hits, steps, warmup)
                refit[lname] = {"refit_ms": trimmed_mean(ts), "closest_mrays_s_after": n / (mc / 1e3) / 1e6,
                                "closest_mode": fc}
            res["trace"] = tr
            res["refit_sah_trees"] = refit
        for bvh in trees.values():
            scion.scion_destroy(bvh)
        out[name] = res
    return out


# ------------------------------------------------------------------ batched (config 4)
def bench_batched(scion, torch, steps, warmup, flush_buf, seed=1004):
    """64 uneven scenes, each with its own rays and autotuned layout: one
    graph-captured batched launch against 64 per-scene plain launches (same
    layouts; and a fixed default layout). Hits must be identical."""
    from paper_2511_15028_gb300 import autotune, scenes
    t0 = time.time()
    wl = scenes.config4_workload(seed=seed)
    gen_s = time.time() - t0
    tuner = autotune.Autotuner()
    rays, chosen = [], []
    t0 = time.time()
    for i, (sc, r) in enumerate(wl):
        d = torch.from_numpy(r).cuda()
        rays.append(d)
        chosen.append(tuner.tune(i, sc.verts, sc.indices, d))
    tune_s = time.time() - t0
    bvhs = [c.bvh for c in chosen]
    params = [c.params for c in chosen]
    batch = scion.Batch(bvhs, rays, params=params)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.launch(stream=stream)
    plain_out = [torch.empty_like(h) for h in batch.hits]

    def plain():
        for b, r, o, p in zip(bvhs, rays, plain_out, params):
            scion.scion_trace_closest(b, r, o, params=p or None)

    default = scion.layout(width=4, box_layout="soa", prim_ref="direct")
    dflt = [scion.scion_build(sc.verts, default, sc.indices) for sc, _ in wl]
    dflt_out = [torch.empty_like(h) for h in batch.hits]

    def plain_default():
        for b, r, o in zip(dflt, rays, dflt_out):
            scion.scion_trace_closest(b, r, o)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush_l2(flush_buf)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return trimmed_mean(ts)

    # the same 64 plain launches captured into one CUDA graph: no host issue
    # cost in the timed region, so the batched launch's gain over it is the
    # traversal's and the load balance's, not the host's
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp, stream=stream):
        plain()
    t_batch = timed(g.replay)
    t_plain_graph = timed(gp.replay)
    t_plain = timed(plain)
    t_dflt = timed(plain_default)
    identical = all(torch.equal(a, b) for a, b in zip(batch.hits, plain_out))
    n_rays = sum(r.shape[0] for r in rays)
    n_tris = sum(sc.n_tris for sc, _ in wl)
    picks = {}
    for c in chosen:
        k = c.name + ("/slot" if c.params else "/ordered")
        picks[k] = picks.get(k, 0) + 1
    info = batch.info()
    return {"scenes": len(wl), "tris": int(n_tris), "rays": int(n_rays),
            "batched_graph_ms": t_batch, "plain_graph_ms": t_plain_graph, "plain_host_ms": t_plain,
            "plain_default_layout_ms": t_dflt,
            "mrays_s_batched": n_rays / (t_batch / 1e3) / 1e6,
            "speedup_vs_plain_graph": t_plain_graph / t_batch, "speedup_vs_plain_host": t_plain / t_batch,
            "speedup_vs_default": t_dflt / t_batch, "batched_scenes": info["batched_scenes"],
            "plain_scenes": info["plain_scenes"],
            "hits_identical": bool(identical), "autotune_picks": picks,
            "gen_s": round(gen_s, 1), "build_and_tune_s": round(tune_s, 1)}


# ------------------------------------------------------------------ differentiation (config 5)
def _fwd_bwd_times(scion, torch, bvh, rays, g, n_verts, steps, warmup, reps, flush_buf=None):
    """Trimmed-mean ms of the forward trace alone and of forward + backward
    (dL/dvertex via FP32 atomics into a zeroed buffer, dL/dray)."""
    n = rays.shape[0]
    hits = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    gv = torch.zeros((n_verts, 3), dtype=torch.float32, device="cuda")
    gr = torch.empty((n, 8), dtype=torch.float32, device="cuda")

    def fwd():
        scion.scion_trace_closest(bvh, rays, hits)

    def fwd_bwd():
        scion.scion_trace_closest(bvh, rays, hits)
        gv.zero_()
        scion.scion_trace_backward(bvh, rays, hits, g, grad_verts=gv, grad_rays=gr)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            if flush_buf is not None:
                flush_l2(flush_buf)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record()
            for _ in range(reps):
                fn()
            b_.record()
            b_.synchronize()
            ts.append(a_.elapsed_time(b_) / reps)
        return trimmed_mean(ts)

    return timed(fwd), timed(fwd_bwd)


def bench_backward(scion, torch, steps, warmup, flush_buf=None):
    """Config-1 scene and rays, L = sum w t + a u + b v: forward alone against
    forward + backward; and the same at the coherent scene's scale (1920 x 1080
    primary rays on 1,373,138 triangles), where launch overhead no longer hides
    the backward kernel."""
    from paper_2511_15028_gb300 import scenes
    lay = scion.layout(width=4, box_layout="soa", prim_ref="direct")
    out = {}
    sc = scenes.config1_scene()
    rays = torch.from_numpy(scenes.config1_rays()).cuda()
    w, a, b = scenes.config5_weights(rays.shape[0])
    g = torch.from_numpy(np.stack([w, a, b], -1)).cuda()
    bvh = scion.scion_build(sc.verts, lay, sc.indices)
    tf, tfb = _fwd_bwd_times(scion, torch, bvh, rays, g, sc.verts.shape[0], steps, warmup, 50)
    n = rays.shape[0]
    out["c5_16384_rays"] = {"rays": n, "fwd_ms": tf, "fwd_bwd_ms": tfb, "mrays_s_fwd": n / (tf / 1e3) / 1e6,
                            "mrays_s_fwd_bwd": n / (tfb / 1e3) / 1e6, "fwd_bwd_over_fwd": tfb / tf,
                            "timing": "50 back-to-back calls per timed step (launch-bound size)"}
    sc2 = scenes.config2_scene()
    rays2 = torch.from_numpy(scenes.config2_primary()).cuda()
    w, a, b = scenes.config5_weights(rays2.shape[0])
    g2 = torch.from_numpy(np.stack([w, a, b], -1)).cuda()
    bvh2 = scion.scion_build(sc2.verts, lay, sc2.indices)
    tf, tfb = _fwd_bwd_times(scion, torch, bvh2, rays2, g2, sc2.verts.shape[0], steps, warmup, 1, flush_buf)
    n = rays2.shape[0]
    out["coherent_primary_2073600_rays"] = {
        "rays": n, "tris": sc2.n_tris, "fwd_ms": tf, "fwd_bwd_ms": tfb, "bwd_ms": tfb - tf,
        "mrays_s_fwd": n / (tf / 1e3) / 1e6, "mrays_s_fwd_bwd": n / (tfb / 1e3) / 1e6,
        "fwd_bwd_over_fwd": tfb / tf, "timing": "one call per timed step, L2 flushed between steps"}
    return out


# ------------------------------------------------------------------ host cost per call
def bench_host(scion, torch, calls=1000, n=1024):
    """Host time per trace call: `calls` back-to-back scion_trace_closest
    calls of n rays (config-1 scene, BVH4), through the C ABI directly
    (ctypes, arguments prepared once) and through the Python binding, timed
    with a host clock; the GPU time of the same loop (CUDA events) is given
    beside it, since a loop faster on the host than on the GPU measures the
    GPU once the launch queue is full."""
    import ctypes

    from paper_2511_15028_gb300 import scenes
    sc = scenes.config1_scene()
    bvh = scion.scion_build(sc.verts, scion.layout(width=4, box_layout="soa", prim_ref="direct"), sc.indices)
    rays = torch.from_numpy(scenes.config1_rays()[:n]).cuda()
    hits = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    L = scion.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (bvh.handle, ctypes.c_void_p(rays.data_ptr()), ctypes.c_uint64(n), ctypes.c_void_p(hits.data_ptr()),
            None, stream)
    out = {"calls": calls, "rays_per_call": n}
    for name, fn in (("c_abi", lambda: L.scion_trace_closest(*args)),
                     ("python", lambda: scion.scion_trace_closest(bvh, rays, hits))):
        for _ in range(50):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        t0 = time.perf_counter()
        for _ in range(calls):
            fn()
        t1 = time.perf_counter()
        b.record()
        b.synchronize()
        out[f"{name}_host_us_per_call"] = round((t1 - t0) / calls * 1e6, 2)
        out[f"{name}_gpu_us_per_call"] = round(a.elapsed_time(b) / calls * 1e3, 2)
    scion.scion_destroy(bvh)
    return out


# ------------------------------------------------------------------ main
def _peaks():
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(pk)) if os.path.exists(pk) else {}
    hbm = peaks.get("hbm_gbs")
    return (hbm, "of measured") if hbm else (6800.0, "of fallback")


def emit(rank, obj):
    """One JSON line on stdout (rank 0 only)."""
    if rank == 0:
        print(json.dumps(obj), flush=True)


def run_section(rank, name, fn, *a, **kw):
    """Run one measurement section and print it as its own JSON line; a
    failing section prints its error and the run goes on."""
    try:
        res = fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported in the section's line
        emit(rank, {"section": name, "error": f"{type(e).__name__}: {e}"})
        return None
    emit(rank, {"section": name, **res})
    return res


SECTIONS = ("incoherent", "batched", "backward", "build", "cpq", "l2", "host")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=9)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--layouts", default="all", help="all | comma-separated sweep names")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fetch", default=None,
                    help="primary,bounce,shadow fetch modes (names of FETCH_MODES / RASTER_MODES), or with "
                         "--section incoherent closest,any; skips the per-layout trials, e.g. to profile "
                         "exactly the modes a plain run chose")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the incoherent, batched, backward, build and closest point sections")
    ap.add_argument("--section", default="all", choices=("all",) + SECTIONS,
                    help="run only one section (e.g. for profiling) and print its line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2511_15028_gb300 import build as native_build
    native_build.build()
    from paper_2511_15028_gb300 import scion

    hbm_peak, peak_src = _peaks()
    if args.section != "all":
        only = None if args.layouts == "all" else args.layouts.split(",")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        fixed = args.fetch.split(",") if args.fetch else None
        fns = {"incoherent": lambda: bench_incoherent(scion, torch, args.steps, args.warmup, hbm_peak, only, fixed),
               "batched": lambda: bench_batched(scion, torch, args.steps, args.warmup, flush),
               "backward": lambda: bench_backward(scion, torch, args.steps, args.warmup, flush),
               "build": lambda: bench_build(scion, torch, args.steps, args.warmup),
               "cpq": lambda: bench_cpq(scion, torch, args.steps, args.warmup, hbm_peak),
               "l2": lambda: measure_l2_peak(scion, torch),
               "host": lambda: bench_host(scion, torch)}
        res = fns[args.section]()
        emit(rank, {"section": args.section, "steps": args.steps, "warmup": args.warmup, **res})
        return

    layouts = scion.sweep_layouts(extended=True)
    if args.layouts != "all":
        keep = args.layouts.split(",")
        layouts = {k: v for k, v in layouts.items() if k in keep}
    first = next(iter(layouts.values()))
    sc, prim, bounce, shadow = make_workload(scion, torch, dev, first)
    n_rays = (prim.shape[0], bounce.shape[0], shadow.shape[0])
    rays = [torch.from_numpy(r).to(dev) for r in (prim, bounce, shadow)]
    outs = [torch.empty((n_rays[0], 4), dtype=torch.int32, device=dev),
            torch.empty((n_rays[1], 4), dtype=torch.int32, device=dev),
            torch.empty((n_rays[2],), dtype=torch.int32, device=dev)]
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)

    # the roof of an L2-resident traversal: this GPU's L2 read bandwidth
    l2 = measure_l2_peak(scion, torch)
    emit(rank, {"section": "l2_peak", **l2})

    results = {}
    sampler = ClockSampler(bus) if rank == 0 else None
    if sampler:
        sampler.start()
    for name, desc in layouts.items():
        bvh = scion.scion_build(sc.verts, desc, sc.indices)
        info = scion.scion_bvh_info(bvh)
        # visit counters for algorithmic bytes (counting kernel, untimed)
        _, cp = scion.scion_trace_stats(bvh, rays[0], 0)
        _, cb = scion.scion_trace_stats(bvh, rays[1], 0)
        _, cs = scion.scion_trace_stats(bvh, rays[2], 1)
        cnt = [c.cpu().numpy() for c in (cp, cb, cs)]
        sn, st = node_load_bytes(desc), tri_load_bytes(desc, True)
        alg = [int(c[3]) * (32 + (16 if q < 2 else 4)) + int(c[0]) * sn + int(c[2]) * st
               for q, c in enumerate(cnt)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        fixed = args.fetch.split(",") if args.fetch else None
        step, per, modes, trials = time_layout(scion, torch, bvh, rays, outs, args.steps, args.warmup, flush_buf,
                                               sampler, fixed)
        ms = trimmed_mean(step.tolist())
        if dist is not None:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        st_status = scion.scion_get_status(bvh)
        per_ms = [trimmed_mean(per[:, i].tolist()) for i in range(3)]
        results[name] = {
            "mrays_s": world * sum(n_rays) / (ms / 1e3) / 1e6,
            "ms_per_step": ms,
            "per_query_ms": {"primary": per_ms[0], "bounce": per_ms[1], "shadow": per_ms[2]},
            "bvh_mb": (info["node_bytes"] + info["prim_bytes"]) / 1e6,
            "node_mb": info["node_bytes"] / 1e6, "n_nodes": info["n_nodes"], "depth": info["depth"],
            "bytes_per_ray": {q: round(alg[i] / max(1, n_rays[i]), 1)
                              for i, q in enumerate(("primary", "bounce", "shadow"))},
            "nodes_per_ray": {q: round(float(cnt[i][0]) / max(1, n_rays[i]), 2)
                              for i, q in enumerate(("primary", "bounce", "shadow"))},
            "tris_per_ray": {q: round(float(cnt[i][2]) / max(1, n_rays[i]), 2)
                             for i, q in enumerate(("primary", "bounce", "shadow"))},
            "alg_bytes": alg, "device_status": st_status,
            "fetch_mode": {"primary": modes[0], "bounce": modes[1], "shadow": modes[2]},
            "fetch_trials_ms": dict(zip(("primary", "bounce", "shadow"), trials)),
        }
        results[name]["_bvh"] = bvh

    clocks = sampler.stop() if sampler else None
    best = max(results, key=lambda k: results[k]["mrays_s"])
    r = results[best]
    # dominant kernel of the best layout's step: the closest-hit kernel (its
    # primary and bounce launches take most of the step); per-launch averages
    tq = r["per_query_ms"]["primary"] + r["per_query_ms"]["bounce"]
    achieved = (r["alg_bytes"][0] + r["alg_bytes"][1]) / (tq / 1e3) / 1e9
    prof = profiled_traffic("coherent", best, "closest")
    l2_peak = l2["peak_gbs"]
    roofline = {"bound": "l2", "achieved": round(achieved, 1), "peak": l2_peak, "unit": "GB/s",
                "frac": round(achieved / l2_peak, 4),
                "traffic": prof["dram_bytes"] if prof else None,
                "l2_traffic": prof["l2_bytes"] if prof else None,
                "traffic_source": prof["source"] if prof else None,
                "kernel": f"trace_kernel closest hit ({best}; primary + bounce launches)",
                "peak_source": "measured live in this run: L2 read bandwidth (section l2_peak)",
                "frac_of_measured_hbm": round(achieved / hbm_peak, 4), "hbm_peak": hbm_peak,
                "hbm_peak_source": peak_src,
                "note": "algorithmic bytes = rays x 48 + nodes visited x node bytes + triangles tested x "
                        "triangle bytes (counting kernel) of one primary and one bounce launch over their "
                        "CUDA-event durations; the BVH fits in L2, so the roof is the L2 read bandwidth; "
                        "traffic / l2_traffic = ncu DRAM / L2 bytes of the same two launches (cold caches)"}
    emit(rank, {"section": "coherent_layouts", "workload": WORKLOAD, "best": best,
                "pareto": pareto({k: (v["bvh_mb"], v["mrays_s"]) for k, v in results.items()}),
                "layouts": {k: {kk: vv for kk, vv in v.items() if kk not in ("alg_bytes", "_bvh")}
                            for k, v in results.items()}})
    # end to end through host buffers, best layout
    fm = r["fetch_mode"]
    e2e_t, bi, bo = e2e_layout(scion, torch, r["_bvh"], (prim, bounce, shadow), args.steps, args.warmup, flush_buf,
                               (fm["primary"], fm["bounce"], fm["shadow"]))
    staged_t, _, _ = e2e_layout(scion, torch, r["_bvh"], (prim, bounce, shadow), args.steps, args.warmup,
                                flush_buf, (fm["primary"], fm["bounce"], fm["shadow"]), zero_copy=False)
    e2e_ms, staged_ms = trimmed_mean(e2e_t), trimmed_mean(staged_t)
    if dist is not None:
        t = torch.tensor([e2e_ms, staged_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms, staged_ms = float(t[0].item()), float(t[1].item())
    e2e = {"value": world * sum(n_rays) / (e2e_ms / 1e3) / 1e6, "unit": "Mrays/s",
           "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": e2e_ms,
           "transfer": "in place: the trace kernels read each step's rays from and write its results to "
                       "pinned host memory over NVLink-C2C (scion.HostTracer(zero_copy=True))",
           "staged_copies": {"value": world * sum(n_rays) / (staged_ms / 1e3) / 1e6, "ms_per_step": staged_ms,
                             "how": "cudaMemcpyAsync of 1M-ray chunks on three streams overlapping the traces"}}
    headline_bvh = r["_bvh"]
    for v in results.values():
        v.pop("_bvh", None)
    del headline_bvh
    if not args.no_extra:
        run_section(rank, "incoherent", bench_incoherent, scion, torch, args.steps, args.warmup, hbm_peak)
        run_section(rank, "batched", bench_batched, scion, torch, args.steps, args.warmup, flush_buf)
        run_section(rank, "backward", bench_backward, scion, torch, args.steps, args.warmup, flush_buf)
        run_section(rank, "build", bench_build, scion, torch, args.steps, args.warmup)
        run_section(rank, "closest_point", bench_cpq, scion, torch, args.steps, args.warmup, hbm_peak)
        run_section(rank, "host", bench_host, scion, torch)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu = cpu_baseline()
    line = {
        "metric": METRIC, "value": r["mrays_s"], "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "layout": best, "rays_per_step": int(sum(n_rays)),
                   "rays": {"primary": n_rays[0], "bounce": n_rays[1], "shadow": n_rays[2]},
                   "fetch_modes": r["fetch_mode"],
                   "l2": "flushed (512 MiB write) between timed steps",
                   "timing": "primary closest hit, then bounce closest hit and shadow any hit concurrently "
                             "on two streams (both come from the primary hits); CUDA events around the step "
                             "on the main stream; trimmed mean of K steps",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "bvh_mb": round(r["bvh_mb"], 2),
        "per_query_ms": {k: round(v, 4) for k, v in r["per_query_ms"].items()},
        "sections": "earlier JSON lines: l2_peak, coherent_layouts (every layout, Pareto front)"
                    + ("" if args.no_extra else ", incoherent, batched, backward, build, closest_point, host"),
    }
    emit(rank, line)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
