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

from paper_1910_13844_gb300.parallel import allreduce_, data_grad_sharded, shard_views


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


class _Prob:
    """Stand-in problem: 5 views of an 8^3 sphere with seeded detector data (kvec as in recon.Problem)."""

    def __init__(self):
        import phantoms as ph
        from oracle import green, model

        self.shape = (8, 8, 8)
        self.st = model.setup_from_optics(self.shape, ph.LAMBDA_UM, ph.ETA_B, ph.VOXEL_UM)
        self.op = model.Operator(self.st)
        self.kvec = ph.cone_directions(5, 0.8) * self.st.kb
        self.ys = [0.01 * ph.complex_normal(self.st.det, 200 + q) for q in range(5)]


def _oracle_data_grad(prob, f, views):
    """CPU stand-in for the library's data_grad: the FP64 oracle's loss and gradient over `views`."""
    from oracle import model

    fn = f.numpy().astype(np.float64)
    uins = [model.plane_wave(prob.shape, prob.st.h, prob.kvec[q]) for q in views]
    ys = [prob.ys[q] for q in views]
    loss = model.loss(prob.op, fn, uins, ys)
    g = model.gradient(prob.op, fn, uins, ys)
    return loss, torch.from_numpy(g)


def _sharded_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import phantoms as ph
    from oracle import green

    prob = _Prob()
    f = torch.from_numpy(green.scattering_potential(ph.sphere(prob.shape, 3.0, 0.05), ph.ETA_B, ph.LAMBDA_UM))
    loss, g = data_grad_sharded(prob, f, data_grad=_oracle_data_grad)
    if rank == 0:
        np.save(os.path.join(out_dir, "sharded_g.npy"), g.numpy())
        np.save(os.path.join(out_dir, "sharded_loss.npy"), np.array([loss]))
        full_loss, full_g = _oracle_data_grad(prob, f, list(range(5)))
        np.save(os.path.join(out_dir, "full_g.npy"), full_g.numpy())
        np.save(os.path.join(out_dir, "full_loss.npy"), np.array([full_loss]))
    dist.barrier()
    dist.destroy_process_group()


def test_data_grad_sharded_reduces_loss_and_gradient_over_ranks(tmp_path):
    world = 2
    mp.start_processes(_sharded_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    g, fg = np.load(tmp_path / "sharded_g.npy"), np.load(tmp_path / "full_g.npy")
    loss, full_loss = float(np.load(tmp_path / "sharded_loss.npy")[0]), float(np.load(tmp_path / "full_loss.npy")[0])
    assert np.linalg.norm(g - fg) <= 1e-12 * np.linalg.norm(fg)
    assert abs(loss - full_loss) <= 1e-12 * abs(full_loss)
