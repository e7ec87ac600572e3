"""The data-parallel training step's exchange on CPU: two gloo ranks each
take their share of the views, form their per-view gradients (the FP64
oracle's adjoint stands in for the GPU backward, which a CPU run cannot
launch) and sum them with sum_gradients; the result must equal the sum over
all views in one process, and sharding must cover every view once."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2604_24994_gb300 import inputs
from paper_2604_24994_gb300.dataparallel import ring_view, shard

PARAMS = ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex")
WORLD = 2


def views():
    return [ring_view(r, 40, 32, radius=3.0, n_ring=4) for r in range(4)]


def upstream(cam, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(cam.n_pixels, 3)), rng.normal(size=cam.n_pixels)


def view_grads(orc, cams, idx):
    tot = None
    for v in idx:
        gC, gT = upstream(cams[v], 100 + v)
        g = orc.render_grad(cams[v], gC, gT)
        tot = g if tot is None else {k: tot[k] + g[k] for k in PARAMS}
    return tot


def _rank(rank, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2604_24994_gb300.dataparallel import sum_gradients
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=WORLD)
    try:
        cams = views()
        mine = shard(range(len(cams)), rank, WORLD)
        g = view_grads(oracle.Oracle(inputs.tiny_scene()), cams, mine)
        t = {k: torch.from_numpy(np.ascontiguousarray(g[k])) for k in PARAMS}
        sum_gradients(t)
        if rank == 0:
            np.savez(out, **{k: t[k].numpy() for k in PARAMS})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_covers_every_view_once():
    for world in (1, 2, 3, 8):
        parts = [shard(range(11), r, world) for r in range(world)]
        assert sorted(sum(parts, [])) == list(range(11))
    with pytest.raises(ValueError):
        shard(range(4), 2, 2)


def test_two_rank_gradient_sum_equals_single_process():
    import torch.multiprocessing as mp

    import oracle
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "g.npz")
        mp.spawn(_rank, args=(free_port(), out), nprocs=WORLD, join=True)
        got = np.load(out)
        cams = views()
        ref = view_grads(oracle.Oracle(inputs.tiny_scene()), cams, range(len(cams)))
        for k in PARAMS:
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-12, atol=1e-12 * np.abs(ref[k]).max())
        # the views really are different: each rank's share alone is not the total
        part = view_grads(oracle.Oracle(inputs.tiny_scene()), cams, shard(range(len(cams)), 0, WORLD))
        assert np.abs(part["pos"] - ref["pos"]).max() > 0
