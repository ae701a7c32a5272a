"""Batched PatchMatch (several reference views in one captured CUDA graph)
and the geometric filter across views it feeds."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ring(mvs_lib, oracle_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=128, H=96, n_src=4, seed=13, baseline_frac=0.1)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    yield sc, ctx, osc
    ctx.close()


REFS = [0, 1, 2, 3]
SRCS = [[1, 2, 3], [0, 2, 4], [0, 1, 3], [0, 2, 4]]


def _separate(mvs, ctx, p):
    out = []
    for r, s in zip(REFS, SRCS):
        pl = np.zeros((96, 128, 4), np.float32)
        co = np.zeros((96, 128), np.float32)
        mvs.mvs_patchmatch(ctx.h, r, s, p, pl, co)
        out.append((pl, co))
    return out


def test_batch_equals_separate_calls_and_replays(ring, mvs_lib):
    sc, ctx, osc = ring
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=2, seed=77)
    ref = _separate(mvs_lib, ctx, p)
    for rep in range(2):                        # capture, then replay of the same graph
        pls = [np.zeros((96, 128, 4), np.float32) for _ in REFS]
        cos = [np.zeros((96, 128), np.float32) for _ in REFS]
        mvs_lib.mvs_patchmatch_batch(ctx.h, REFS, SRCS, p, pls, cos)
        for (a_pl, a_co), b_pl, b_co in zip(ref, pls, cos):
            assert np.array_equal(a_pl, b_pl) and np.array_equal(a_co, b_co)


def test_batch_device_buffers_and_autotuned_layout(ring, mvs_lib):
    import torch
    sc, ctx, osc = ring
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=2, seed=78)
    ref = _separate(mvs_lib, ctx, p)
    q = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=2, seed=78, lanes_per_pixel=-1)
    pls = [torch.zeros((96, 128, 4), dtype=torch.float32, device="cuda") for _ in REFS]
    cos = [torch.zeros((96, 128), dtype=torch.float32, device="cuda") for _ in REFS]
    mvs_lib.mvs_patchmatch_batch(ctx.h, REFS, SRCS, q, pls, cos)
    torch.cuda.synchronize()
    for (a_pl, a_co), b_pl, b_co in zip(ref, pls, cos):
        b_pl, b_co = b_pl.cpu().numpy(), b_co.cpu().numpy()
        # another work layout only reorders float additions inside a group:
        # the same decisions almost everywhere, costs equal to rounding
        same = (np.abs(a_pl[..., 3] - b_pl[..., 3]) <= 1e-5 * a_pl[..., 3]) & \
               (np.abs(a_pl[..., :3] - b_pl[..., :3]).max(-1) <= 1e-5)
        assert same.mean() > 0.97
        # each layout is within 1e-4 of the FP64 oracle, so within 2e-4 of each other
        assert np.abs(a_co - b_co)[same].max() < 2e-4


def test_batch_rejects_repeated_reference(ring, mvs_lib):
    sc, ctx, osc = ring
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=1)
    pls = [np.zeros((96, 128, 4), np.float32) for _ in range(2)]
    cos = [np.zeros((96, 128), np.float32) for _ in range(2)]
    with pytest.raises(mvs_lib.MvsError) as e:
        mvs_lib.mvs_patchmatch_batch(ctx.h, [1, 1], [[0, 2, 3], [0, 2, 3]], p, pls, cos)
    assert e.value.status == mvs_lib.MVS_EINVAL


def test_geo_filter_across_batched_views(ring, mvs_lib, oracle_lib):
    """After a batched run every view has a map; the GPU filter of each view
    against its sources matches the oracle's filter on the same maps."""
    sc, ctx, osc = ring
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=3, seed=79)
    pls = [np.zeros((96, 128, 4), np.float32) for _ in REFS]
    cos = [np.zeros((96, 128), np.float32) for _ in REFS]
    mvs_lib.mvs_patchmatch_batch(ctx.h, REFS, SRCS, p, pls, cos)
    maps = {r: pl.astype(np.float64) for r, pl in zip(REFS, pls)}
    fp = mvs_lib.FilterParams(min_consistent=1)      # three sources: ask for at least one
    for r in REFS:
        others = [v for v in REFS if v != r]
        keep = np.zeros((96, 128), np.uint8)
        cnt = np.zeros((96, 128), np.int32)
        mvs_lib.mvs_geo_filter(ctx.h, r, others, fp, keep, cnt)
        okeep, ocnt, mg = oracle_lib.geo_filter(osc, r, others, maps, min_consistent=1, with_margin=True)
        assert keep.mean() > 0.3
        firm = mg >= 1.0       # outside the oracle's fragile band: identical
        assert np.array_equal(cnt[firm], ocnt[firm]) and np.array_equal(keep[firm], okeep[firm])
        assert firm.mean() > 0.99
        gt = sc.gt_depth if r == 0 else None
        if gt is not None:     # kept pixels are mostly right
            good = np.abs(pls[0][..., 3] - gt) / gt < 0.01
            assert good[keep == 1].mean() > 0.9


def test_batch_takes_back_to_back_proposals(ring, mvs_lib):
    """Learned proposals in the batched graph: every reference's H x W x K
    planes back to back in refs order give the maps of separate
    mvs_patchmatch calls with each view's own proposals, bit for bit, on
    capture and on replay."""
    import torch
    sc, ctx, osc = ring
    H, W, K = 96, 128, 4
    rng = np.random.default_rng(4)
    props = []
    for r in REFS:
        n = rng.normal(0, 1, (H, W, K, 3))
        n[..., 2] = -np.abs(n[..., 2]) - 0.5
        n /= np.linalg.norm(n, axis=-1, keepdims=True)
        props.append(np.concatenate([n, rng.uniform(2.5, 7.5, (H, W, K, 1))], -1).astype(np.float32))
    d_props = [torch.from_numpy(p).cuda() for p in props]
    base = dict(win_radius=5.0, win_samples=6, iters=2, seed=31, n_prop=K)
    sep = []
    for r, s, dp in zip(REFS, SRCS, d_props):
        pl = np.zeros((H, W, 4), np.float32)
        co = np.zeros((H, W), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, r, s, mvs_lib.PMParams(**base, proposals=dp), pl, co)
        sep.append((pl, co))
    both = torch.cat([dp.reshape(-1) for dp in d_props])
    q = mvs_lib.PMParams(**base, proposals=both)
    for _ in range(2):
        pls = [np.zeros((H, W, 4), np.float32) for _ in REFS]
        cos = [np.zeros((H, W), np.float32) for _ in REFS]
        mvs_lib.mvs_patchmatch_batch(ctx.h, REFS, SRCS, q, pls, cos)
        for (a_pl, a_co), b_pl, b_co in zip(sep, pls, cos):
            assert np.array_equal(a_pl, b_pl) and np.array_equal(a_co, b_co)
    # the proposals matter: without them the maps differ
    plain = _separate(mvs_lib, ctx, mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=2, seed=31))
    assert any(not np.array_equal(a[0], b[0]) for a, b in zip(plain, sep))
