"""Multi-rank paths on CPU (gloo, world size 2).

Walks are independent and keyed by their global walk id, so sharding the
query points across ranks (each rank running its points with the matching
walk-id base) and summing per-point partial sums reproduces the unsharded
result bit for bit, for walks on spheres and for walks on stars with
Neumann data (whose per-step element draw is keyed by the walk id too).
Also checks the bench's rank aggregation (max time, sum of walk-steps).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _scene(name):
    from paper_2405_12964_gb300 import scenes
    if name == "disk":
        return scenes.disk_scene("screened_1", n_query=10)
    return scenes.neumann_data_box_scene(2, n_query=10)


def _worker(rank, world, port, q, name):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2405_12964_gb300 import scenes
        from tests.helpers import to_oracle
        import bench
        sc = _scene(name)
        W = 48
        n = sc.query.shape[0]
        bounds = np.linspace(0, n, world + 1).astype(int)
        p0, p1 = bounds[rank], bounds[rank + 1]
        o = oracle.run_walks(to_oracle(sc), sc.query[p0:p1], W, differential=True, walk_id_base=int(p0) * W)
        sums = np.zeros((n, 1 + sc.n_param))
        sums[p0:p1, 0] = o["u_hat"].reshape(p1 - p0, W).sum(1)
        sums[p0:p1, 1:] = o["udot"].reshape(p1 - p0, W, -1).sum(1)
        t = torch.tensor(sums)
        dist.all_reduce(t)
        steps = int(o["steps"].clip(min=0).sum())
        tmax, steps_all = bench.aggregate_ranks(0.5 + rank, steps, dist, "cpu")
        q.put((rank, t.numpy(), tmax, steps_all, steps))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["disk", "neumann_data_box"])
def test_sharded_walks_reduce_to_the_unsharded_result(name):
    import oracle
    from paper_2405_12964_gb300 import scenes
    from tests.helpers import to_oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, name)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    sc = _scene(name)
    W = 48
    o = oracle.run_walks(to_oracle(sc), sc.query, W, differential=True)
    want = np.zeros((10, 1 + sc.n_param))
    want[:, 0] = o["u_hat"].reshape(10, W).sum(1)
    want[:, 1:] = o["udot"].reshape(10, W, -1).sum(1)
    for r in res:
        assert np.array_equal(r[1], want)          # bit-exact
        assert r[2] == 1.5                         # max over ranks
        assert r[3] == res[0][4] + res[1][4]       # sum of walk-steps
