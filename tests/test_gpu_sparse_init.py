"""Depth initialisation from sparse features (Sec. III-B) on the GPU against
the FP64 oracle: the per-pixel ranges bit for bit (the library rounds the
feature depths to float) wherever the closest-feature choice is firm, with
the pixels whose choice lies within BAND_PX of a boundary counted, printed
and bounded; the initial state within the initialisation tolerances, and
the faster convergence the paper argues for."""
import copy

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the library keeps feature positions in float (< 7.6e-6 px of rounding at
# these sizes) and distances in float (~1e-6 px); the band is ten times that
BAND_PX = 1e-4


def _masks(vis):
    m = np.zeros(len(vis), np.uint64)
    for v in range(vis.shape[1]):
        m |= vis[:, v].astype(np.uint64) << np.uint64(v)
    return m


@pytest.fixture(scope="module")
def sparse_scene(mvs_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=4, seed=13, baseline_frac=0.1)
    sp = scenes.sparse_points(sc, 1500, seed=2)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    yield sc, sp, ctx
    ctx.close()


def _gpu_range(mvs_lib, ctx, sp, ref, H, W, device=False):
    import torch
    X = np.ascontiguousarray(sp["X"], np.float64)
    m = _masks(sp["vis"])
    rep = np.ascontiguousarray(sp["reproj"], np.float64)
    obs = np.ascontiguousarray(sp["obs"][:, ref], np.float64)
    if device:
        out = torch.zeros((H, W, 2), dtype=torch.float32, device="cuda")
        mvs_lib.mvs_sparse_depth_range(ctx.h, ref, torch.from_numpy(X).cuda(), torch.from_numpy(m.view(np.int64)).cuda(),
                                       torch.from_numpy(rep).cuda(), torch.from_numpy(obs).cuda(), out)
        return out
    out = np.zeros((H, W, 2), np.float32)
    mvs_lib.mvs_sparse_depth_range(ctx.h, ref, X, m, rep, obs, out)
    return out


@pytest.mark.parametrize("ref", [0, 2])
def test_ranges_equal_oracle(sparse_scene, mvs_lib, oracle_lib, ref):
    sc, sp, ctx = sparse_scene
    H, W = sc.images[ref].shape
    g = _gpu_range(mvs_lib, ctx, sp, ref, H, W)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    uv, dep = oracle_lib.sparse_features(osc, ref, sp["X"], sp["vis"], sp["reproj"], sp["obs"][:, ref])
    o, frag = oracle_lib.sparse_range(W, H, uv, dep, d_lo=2.0, d_hi=8.0, band_px=BAND_PX, fragile=True)
    print(f"sparse ranges: {frag.sum()} of {frag.size} pixels fragile ({frag.mean():.2e})")
    assert frag.mean() < 0.01
    firm = ~frag
    o32 = o.astype(np.float32)
    assert np.array_equal(np.isnan(g[firm]), np.isnan(o32[firm]))
    ok = ~np.isnan(o32[firm])
    assert np.array_equal(g[firm][ok], o32[firm][ok])
    # a fragile pixel still gets a valid range
    gf = g[frag]
    gf = gf[~np.isnan(gf[:, 0])]
    assert ((gf[:, 0] <= gf[:, 1]) & (gf[:, 0] >= 2.0) & (gf[:, 1] <= 8.0)).all()
    assert (~np.isnan(o[..., 0])).mean() > 0.5      # most pixels get a range
    # device buffers give the same ranges
    d = _gpu_range(mvs_lib, ctx, sp, ref, H, W, device=True).cpu().numpy()
    assert np.array_equal(np.isnan(d), np.isnan(g)) and np.array_equal(d[~np.isnan(d)], g[~np.isnan(g)])


def test_initial_state_matches_oracle(sparse_scene, mvs_lib, oracle_lib):
    import torch
    sc, sp, ctx = sparse_scene
    H, W = sc.images[0].shape
    rng = _gpu_range(mvs_lib, ctx, sp, 0, H, W, device=True)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=0, seed=21, init_mode=mvs_lib.MVS_INIT_RANGE,
                         init_range=rng)
    pl = np.zeros((H, W, 4), np.float32)
    co = np.zeros((H, W), np.float32)
    mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2, 3, 4], p, pl, co)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    q = copy.copy(p)
    q.init_range = None
    opl, oco = oracle_lib.init(osc, 0, [1, 2, 3, 4], q, init_range=rng.cpu().numpy())
    assert np.abs(pl[..., 3] - opl[..., 3]).max() < 1e-5 * 8
    assert np.abs(pl[..., :3] - opl[..., :3]).max() < 1e-5
    assert (np.abs(co - oco) <= 1e-4).mean() > 0.995
    # the depths lie in their ranges
    r = rng.cpu().numpy()
    has = ~np.isnan(r[..., 0])
    assert ((pl[..., 3] >= r[..., 0] - 1e-6) & (pl[..., 3] <= r[..., 1] + 1e-6))[has].all()


def test_sparse_initialisation_converges_faster(sparse_scene, mvs_lib):
    sc, sp, ctx = sparse_scene
    H, W = sc.images[0].shape
    rng = _gpu_range(mvs_lib, ctx, sp, 0, H, W, device=True)
    gt = sc.gt_depth
    tex = sc.gt_textured

    def comp(params):
        pl = np.zeros((H, W, 4), np.float32)
        co = np.zeros((H, W), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2, 3, 4], params, pl, co)
        return float((np.abs(pl[..., 3] - gt) <= 0.01 * gt)[tex].mean())

    base = dict(win_radius=5.0, win_samples=6, iters=1, seed=5)
    plain = comp(mvs_lib.PMParams(**base))
    sparse = comp(mvs_lib.PMParams(**base, init_mode=mvs_lib.MVS_INIT_RANGE, init_range=rng))
    assert sparse > plain


def test_ranges_must_be_device_memory(sparse_scene, mvs_lib):
    sc, sp, ctx = sparse_scene
    H, W = sc.images[0].shape
    host = np.zeros((H, W, 2), np.float32)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=0, init_mode=mvs_lib.MVS_INIT_RANGE, init_range=host)
    with pytest.raises(mvs_lib.MvsError):
        mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2], p, np.zeros((H, W, 4), np.float32), np.zeros((H, W), np.float32))
    with pytest.raises(mvs_lib.MvsError):
        mvs_lib.mvs_patchmatch_batch(ctx.h, [0], [[1, 2]], p, [np.zeros((H, W, 4), np.float32)],
                                     [np.zeros((H, W), np.float32)])


def test_batch_takes_back_to_back_ranges(sparse_scene, mvs_lib):
    """The batched graph with every reference's ranges back to back in refs
    order gives the maps of separate mvs_patchmatch calls, bit for bit."""
    import torch
    sc, sp, ctx = sparse_scene
    H, W = sc.images[0].shape
    refs, srcs = [2, 0], [[0, 1, 3, 4], [1, 2, 3, 4]]
    rngs = [_gpu_range(mvs_lib, ctx, sp, r, H, W, device=True) for r in refs]
    sep = []
    for r, s, g in zip(refs, srcs, rngs):
        p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=1, seed=12, init_mode=mvs_lib.MVS_INIT_RANGE,
                             init_range=g)
        pl = np.zeros((H, W, 4), np.float32)
        co = np.zeros((H, W), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, r, s, p, pl, co)
        sep.append((pl, co))
    both = torch.cat([g.reshape(-1) for g in rngs])
    q = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=1, seed=12, init_mode=mvs_lib.MVS_INIT_RANGE,
                         init_range=both)
    for _ in range(2):      # capture, then replay
        pls = [np.zeros((H, W, 4), np.float32) for _ in refs]
        cos = [np.zeros((H, W), np.float32) for _ in refs]
        mvs_lib.mvs_patchmatch_batch(ctx.h, refs, srcs, q, pls, cos)
        for (a_pl, a_co), b_pl, b_co in zip(sep, pls, cos):
            assert np.array_equal(a_pl, b_pl) and np.array_equal(a_co, b_co)
    # the two views' ranges differ, so taking one view's ranges for both would fail
    assert not torch.equal(rngs[0].isnan(), rngs[1].isnan()) or not torch.equal(rngs[0].nan_to_num(),
                                                                                   rngs[1].nan_to_num())


def test_no_features_keeps_the_random_initialisation(sparse_scene, mvs_lib):
    import torch
    sc, sp, ctx = sparse_scene
    H, W = sc.images[0].shape
    empty = {k: v[:0] for k, v in sp.items()}
    rng = _gpu_range(mvs_lib, ctx, empty, 0, H, W, device=True)
    assert torch.isnan(rng).all()
    base = dict(win_radius=5.0, win_samples=6, iters=0, seed=17)
    outs = []
    for extra in ({}, dict(init_mode=mvs_lib.MVS_INIT_RANGE, init_range=rng)):
        pl = np.zeros((H, W, 4), np.float32)
        co = np.zeros((H, W), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2, 3, 4], mvs_lib.PMParams(**base, **extra), pl, co)
        outs.append((pl, co))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
