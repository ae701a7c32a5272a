"""World-size-2 gloo test of the multi-rank host logic (view sharding and the
plane-map exchange before the geometric filter)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2104_06165_gb300.dist import assign_views, exchange_plane_maps, owner_of


def test_assignment_balances_pixels():
    counts = [3072 * 2048] * 8 + [2048 * 1365] * 8 + [1536 * 1024] * 8
    parts = assign_views(counts, 4)
    assert sorted(v for p in parts for v in p) == list(range(24))
    loads = [sum(counts[v] for v in p) for p in parts]
    assert max(loads) - min(loads) <= 1536 * 1024
    assert assign_views([5, 5], 1) == [[0, 1]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, shapes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = assign_views([h * w for h, w in shapes], world)
        mine = {}
        for v in parts[rank]:
            H, W = shapes[v]
            mine[v] = torch.full((H, W, 4), float(v)) + torch.arange(H * W * 4, dtype=torch.float32).reshape(H, W, 4)
        allm = exchange_plane_maps(mine, shapes, parts)
        ok = all(torch.equal(allm[v], torch.full(shapes[v] + (4,), float(v)) +
                             torch.arange(shapes[v][0] * shapes[v][1] * 4, dtype=torch.float32).reshape(
                                 shapes[v] + (4,))) for v in range(len(shapes)))
        q.put((rank, ok, sorted(allm)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world, shapes", [(2, [(6, 8), (5, 7), (6, 8), (3, 4), (4, 4)]),
                                           (3, [(6, 8), (5, 7)])])
def test_gloo_exchange(world, shapes):
    """World 2 with five views, and world 3 with two views (one rank owns
    none and receives both)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, shapes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, views in res:
        assert ok and views == list(range(len(shapes)))
    assert set(owner_of(assign_views([48, 35, 48, 12, 16], 2)).values()) == {0, 1}


def _sub_worker(rank, world, port, shapes, q):
    """Ranks 1 and 2 of a world of 3 exchange in a subgroup: the owner's
    group rank is mapped to its global rank for the broadcast."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = dist.new_group([1, 2])
        if rank in (1, 2):
            parts = assign_views([h * w for h, w in shapes], 2)
            gr = dist.get_rank(g)
            mine = {v: torch.full(shapes[v] + (4,), float(10 * v + 1)) for v in parts[gr]}
            allm = exchange_plane_maps(mine, shapes, parts, group=g)
            ok = all(torch.equal(allm[v], torch.full(shapes[v] + (4,), float(10 * v + 1))) for v in range(len(shapes)))
            q.put((rank, ok))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gloo_subgroup_exchange():
    shapes = [(6, 8), (5, 7), (4, 4)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sub_worker, args=(r, 3, port, shapes, q)) for r in range(3)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(1, True), (2, True)]


# --------------------------------------------------------------------------
# the sharded depth-map stage on gloo ranks with the FP64 oracle as the
# per-rank compute: views by assign_views, the exchange, the filter on the
# received maps, against one process doing everything
# --------------------------------------------------------------------------
def _small_scene():
    from paper_2104_06165_gb300 import scenes
    return scenes.make_scene(W=40, H=30, n_src=3, seed=4, baseline_frac=0.1)


class _P:
    def __init__(self):
        self.win_radius, self.win_samples = 5.0, 6
        self.sigma_s, self.sigma_c = 5.0, 0.2
        self.d_lo, self.d_hi, self.seed = 2.0, 8.0, 3


def _oracle_maps(osc, views, n):
    import oracle
    out = {}
    for v in views:
        pl, _ = oracle.patchmatch(osc, v, [u for u in range(n) if u != v], _P(), 1)
        out[v] = pl
    return out


def _sharded_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np
        import oracle
        sc = _small_scene()
        n = sc.n_views
        osc = oracle.Scene(sc.K, sc.R, sc.t, sc.images)
        shapes = [im.shape for im in sc.images]
        parts = assign_views([h * w for h, w in shapes], world)
        mine = _oracle_maps(osc, parts[rank], n)
        # plane maps travel as float32, the library's format
        allm = exchange_plane_maps({v: torch.from_numpy(m.astype(np.float32)) for v, m in mine.items()}, shapes,
                                   parts)
        planes = {v: t.numpy().astype(np.float64) for v, t in allm.items()}
        keeps = {v: oracle.geo_filter(osc, v, [u for u in range(n) if u != v], planes)[0] for v in parts[rank]}
        q.put((rank, keeps))
    finally:
        dist.destroy_process_group()


def test_gloo_sharded_filter_equals_one_process():
    import numpy as np
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = _small_scene()
    n = sc.n_views
    osc = oracle.Scene(sc.K, sc.R, sc.t, sc.images)
    planes = {v: m.astype(np.float32).astype(np.float64) for v, m in _oracle_maps(osc, range(n), n).items()}
    got = {v: k for r in res.values() for v, k in r.items()}
    assert sorted(got) == list(range(n)) and set(res[0]).isdisjoint(res[1])
    for v in range(n):
        ref = oracle.geo_filter(osc, v, [u for u in range(n) if u != v], planes)[0]
        assert np.array_equal(got[v], ref)
    assert any(k.any() for k in got.values())
