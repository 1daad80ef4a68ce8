"""Two CPU ranks (gloo): views sharded over ranks, per-rank FP64 adjoints of
the oracle summed with the package's gradient reduction, against one rank
doing everything, for an isotropic and an anisotropic pyramid.  Exercises
the exchange the sharded path needs."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import vct_synth as vs
from paper_2104_00618_gb300.sharding import reduce_gradient, shard


def _case():
    gt = vs.box_scene(8, 3, 91, room=True)
    rng = np.random.default_rng(92)
    views = [vs.interior_view(gt, 6, 5, rng, with_roughness=False) for _ in range(5)]
    dirs, w = vs.cone_table_ring6()
    prm = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                          spec_aperture_min=math.radians(20), occ_enable=True,
                          light=gt["light"], t_max=0.6)
    learn = np.random.default_rng(93).uniform(0.0, 0.3, (8, 8, 8, 4))
    return gt, views, prm, learn


def _grad(views, prm, learn, gt, aniso=False):
    build = oracle.build_mips_aniso if aniso else oracle.build_mips
    P, Pgt = build(learn), build(gt["grid"])
    g = np.zeros(learn.shape)
    for v in views:
        r, t = oracle.trace(P, v, prm), oracle.trace(Pgt, v, prm)
        g += oracle.trace_backward(P, v, prm, r["D"] - t["D"], r["S"] - t["S"],
                                   r["Vis"] - t["Vis"])
    return g


def _worker(rank, world, port, out_path, aniso):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    gt, views, prm, learn = _case()
    mine = shard(views, rank, world)
    g = torch.from_numpy(_grad(mine, prm, learn, gt, aniso))
    reduce_gradient(g)
    if rank == 0:
        np.save(out_path, g.numpy())
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_every_item_once():
    items = list(range(11))
    parts = [shard(items, r, 4) for r in range(4)]
    assert sum(parts, []) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


@pytest.mark.parametrize("aniso", [False, True])
def test_two_rank_gradient_equals_single_rank(tmp_path, aniso):
    oracle.build()  # compile before spawning
    out = str(tmp_path / "g.npy")
    mp.spawn(_worker, args=(2, _free_port(), out, aniso), nprocs=2, join=True)
    gt, views, prm, learn = _case()
    ref = _grad(views, prm, learn, gt, aniso)
    got = np.load(out)
    assert np.abs(got).max() > 0
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())
