"""Data-parallel differentiation over two ranks (gloo, CPU): each rank differentiates its
share of the views and one all-reduce sums the parameter gradients; the sum must equal the
gradient of all views on one rank, and the plane gradients stay with their views. The
per-rank gradient here is the oracle's analytic FP64 gradient (no GPU)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    from paper_2506_20202_gb300 import scenes
    sc = scenes.gradient_scene(40, seed=11, sh_degree=1)
    views = []
    for k in range(5):   # 5 views: ranks get 3 and 2
        a = 2.0 * np.pi * k / 5
        cam = scenes.look_at_camera((2.8 * np.sin(a), -0.4, -2.8 * np.cos(a)), (0.0, 0.0, 0.0), 40 + 8 * k, 36, 60.0)
        pl = scenes.Plane(np.float32(scenes.random_unit_normal(20 + k)), 0.03 * k - 0.05, 3.0, scenes.MODE_RARA)
        views.append((cam, pl))
    rng = np.random.default_rng(3)
    weights = [rng.standard_normal((3, c.height, c.width)) for c, _ in views]
    return sc, views, weights


def _local_fn(sc, views, weights):
    from oracle import grad as ograd

    def fn(idx):
        loss = 0.0
        grads = {k: torch.zeros(getattr(sc, k).shape, dtype=torch.float64) for k in ograd.PARAMS}
        planes = {}
        for v in idx:
            cam, pl = views[v]
            g = ograd.render_and_grad(sc, cam, pl, (0.0, 0.0, 0.0), weights[v])
            loss += float(np.sum(weights[v] * g["image"]))
            for k in ograd.PARAMS:
                grads[k] += torch.from_numpy(g[k])
            planes[v] = g["plane"]
        return torch.tensor(loss, dtype=torch.float64), grads, planes
    return fn


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2506_20202_gb300 import dp
        sc, views, weights = _workload()
        res = dp.data_parallel_gradients(_local_fn(sc, views, weights), len(views), rank, world)
        q.put((rank, float(res.loss), {k: v.numpy() for k, v in res.grads.items()}, res.plane_grads, res.views))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_to_the_single_rank_gradient():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc, views, weights = _workload()
    loss, full, planes = _local_fn(sc, views, weights)(list(range(len(views))))
    assert [g[4] for g in got] == [[0, 2, 4], [1, 3]]
    for rank, l, grads, pg, mine in got:
        assert l == pytest.approx(float(loss), rel=1e-12)
        for k, v in full.items():
            assert np.allclose(grads[k], v.numpy(), rtol=1e-10, atol=1e-13), (rank, k)
        for v in mine:                       # each view's plane gradient stays on its rank
            assert np.array_equal(pg[v], planes[v])
        assert set(pg) == set(mine)
    assert np.linalg.norm(full["means"].numpy()) > 0


def test_sharding_and_single_rank_no_op():
    from paper_2506_20202_gb300 import dp
    assert dp.shard_views(7, 0, 3) == [0, 3, 6] and dp.shard_views(7, 2, 3) == [2, 5]
    assert sorted(sum((dp.shard_views(64, r, 8) for r in range(8)), [])) == list(range(64))
    with pytest.raises(ValueError):
        dp.shard_views(4, 2, 2)
    t = [torch.ones(3)]
    assert dp.allreduce_sum(t)[0].tolist() == [1.0, 1.0, 1.0]     # no process group: unchanged
