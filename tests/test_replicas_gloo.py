"""Host-side multi-rank logic on CPU (gloo, world size 2): ray shards cover
the batch exactly once, gathered shards reproduce the whole-batch result, the
vertex-gradient all-reduce equals the single-process sum, and the timing
reduction takes the slowest rank. The per-shard work here is the CPU oracle
(the GPU kernels are covered by the -m gpu tests)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_15028_gb300 import replicas


def test_shard_range_partitions():
    for n in (0, 1, 5, 16, 17, 1000003):
        for w in (1, 2, 3, 8):
            got = [replicas.shard_range(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outq):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2511_15028_gb300 import scenes
        sc = scenes.config1_scene()
        rays = scenes.config1_rays()
        tris = sc.triangles()
        n = rays.shape[0]
        b, e = replicas.shard_range(n, rank, world)
        hits = oracle.closest_brute(tris, rays[b:e], threads=1)
        local = torch.from_numpy(hits.view(np.int32).reshape(-1, 4).copy())
        full = replicas.gather_shards(local, n)
        w, a, bb = scenes.config5_weights(n)
        g = np.stack([w, a, bb], -1)[b:e]
        gv, _ = oracle.grad(tris, sc.indices, sc.verts.shape[0], rays[b:e], hits, g)
        gsum = replicas.allreduce_vertex_grads(torch.from_numpy(gv))
        slowest = replicas.max_over_ranks(1.0 + rank)
        if rank == 0:
            outq.put((full.numpy().tobytes(), gsum.numpy().tobytes(), slowest))
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_and_gradient_allreduce(oracle_mod):
    import oracle
    from paper_2511_15028_gb300 import scenes
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full, gsum, slowest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = scenes.config1_scene()
    rays = scenes.config1_rays()
    tris = sc.triangles()
    ref = oracle.closest_brute(tris, rays)
    assert full == ref.view(np.int32).reshape(-1, 4).tobytes()
    w, a, bb = scenes.config5_weights(rays.shape[0])
    gv, _ = oracle.grad(tris, sc.indices, sc.verts.shape[0], rays, ref, np.stack([w, a, bb], -1))
    got = np.frombuffer(gsum, np.float64).reshape(-1, 3)
    np.testing.assert_allclose(got, gv, rtol=1e-12, atol=1e-12)
    assert slowest == 2.0
