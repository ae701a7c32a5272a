"""The sharded depth-map stage through the library (dist.filter_sharded):
two gloo ranks, each on the same GPU in its own process, run their share
of the views as one batched PatchMatch call, exchange the plane maps through
host memory, store the received maps with mvs_set_depth_map and filter their
own views.  Keep masks and maps equal those of one process that runs every
view, bit for bit (the kernels are deterministic and the maps do not depend
on which views share a batch)."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scene():
    from paper_2104_06165_gb300 import scenes
    return scenes.make_scene(W=96, H=72, n_src=4, seed=21, baseline_frac=0.1)


def _params(mvs):
    return mvs.PMParams(win_radius=5.0, win_samples=6, iters=2, seed=8, lanes_per_pixel=4)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    from paper_2104_06165_gb300 import dist as pdist, mvs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        sc = _scene()
        n = sc.n_views
        with mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream()) as ctx:
            keeps, planes = pdist.filter_sharded(mvs, ctx, [im.shape for im in sc.images],
                                                 [[u for u in range(n) if u != v] for v in range(n)], _params(mvs),
                                                 mvs.FilterParams())
            torch.cuda.synchronize()
            q.put((rank, {v: k.cpu().numpy() for v, k in keeps.items()},
                   {v: p.cpu().numpy() for v, p in planes.items()}))
    finally:
        dist.destroy_process_group()


def test_sharded_filter_equals_one_process(mvs_lib):
    import multiprocessing as mp
    import torch
    ctxm = mp.get_context("spawn")
    q = ctxm.Queue()
    port = _free_port()
    procs = [ctxm.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, k, pl = q.get(timeout=600)
        res[r] = (k, pl)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sc = _scene()
    n = sc.n_views
    srcs_of = [[u for u in range(n) if u != v] for v in range(n)]
    with mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream()) as ctx:
        H, W = sc.images[0].shape
        planes = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(n)]
        costs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(n)]
        mvs_lib.mvs_patchmatch_batch(ctx.h, list(range(n)), srcs_of, _params(mvs_lib), planes, costs)
        keeps = []
        for v in range(n):
            k = torch.empty((H, W), dtype=torch.uint8, device="cuda")
            mvs_lib.mvs_geo_filter(ctx.h, v, srcs_of[v], mvs_lib.FilterParams(), k)
            keeps.append(k.cpu().numpy())
        planes = [p.cpu().numpy() for p in planes]
    owned = {v: r for r, (k, _) in res.items() for v in k}
    assert sorted(owned) == list(range(n)) and len(set(owned.values())) == 2
    for v, r in owned.items():
        k, pl = res[r][0][v], res[r][1][v]
        assert np.array_equal(pl, planes[v]), f"view {v}: plane map"
        assert np.array_equal(k, keeps[v]), f"view {v}: keep mask"
    assert sum(k.sum() for k in keeps) > 0
