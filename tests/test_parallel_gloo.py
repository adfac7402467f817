"""Multi-rank logic on CPU (gloo, world size 2): view sharding and the gradient all-reduce.

Each rank computes the FP64 oracle gradient of eq. prob for its shard of the views; the summed
gradient must equal the single-process gradient over all views.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1910_13844_gb300.parallel import allreduce_, shard_views


def test_shards_cover_every_view_once():
    for n in (1, 5, 60, 61):
        for world in (1, 2, 3, 8):
            got = [list(shard_views(n, world, r)) for r in range(world)]
            flat = [v for g in got for v in g]
            assert flat == list(range(n))
            sizes = [len(g) for g in got]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import phantoms as ph
    from oracle import green, model

    shape = (8, 8, 8)
    st = model.setup_from_optics(shape, ph.LAMBDA_UM, ph.ETA_B, ph.VOXEL_UM)
    op = model.Operator(st)
    f = green.scattering_potential(ph.sphere(shape, 3.0, 0.05), ph.ETA_B, ph.LAMBDA_UM)
    kvecs = ph.cone_directions(5, 0.8) * st.kb
    ys = [0.01 * ph.complex_normal(st.det, 100 + q) for q in range(5)]
    mine = list(shard_views(5, world, rank))
    g = model.gradient(op, f, [model.plane_wave(shape, st.h, kvecs[q]) for q in mine], [ys[q] for q in mine])
    t = torch.from_numpy(g)
    allreduce_(t)
    if rank == 0:
        np.save(os.path.join(out_dir, "sharded.npy"), t.numpy())
        full = model.gradient(op, f, [model.plane_wave(shape, st.h, k) for k in kvecs], ys)
        np.save(os.path.join(out_dir, "full.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_gradient_equals_full_gradient(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    a = np.load(tmp_path / "sharded.npy")
    b = np.load(tmp_path / "full.npy")
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
