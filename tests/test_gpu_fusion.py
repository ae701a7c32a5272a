"""Depth-map fusion (Sec. III-F) on the GPU (single precision) against the
FP64 oracle.  A decision within rounding of its boundary — a projection
whose u + 1/2 or v + 1/2 lies within BAND_PX of an integer, or a distance
within BAND_REL of the 1 % threshold — may go either way in FP32; the
oracle counts those and follows the library's choice there (given as the
per-pixel point index), taking every other decision itself.  The number of
points, the emitting pixels, every pixel's point and the merge counts then
agree exactly, the points within FP32 rounding, and the fragile fraction is
printed and bounded."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# FP32 moves a projection by about f 1e-6 / z (< 1e-4 px here) and a
# distance by about 1e-4 of the threshold; the bands are ten times that
BAND_PX, BAND_REL = 1e-3, 1e-3


def _close(pts, opts):
    """FP32 points against FP64 ones: counts equal, coordinates within
    rounding of the back-projection chain."""
    return np.array_equal(pts[:, 3], opts[:, 3]) and np.allclose(pts[:, :3], opts[:, :3], rtol=4e-6, atol=1e-5)

F, CX, CY = 100.0, 11.5, 3.5
W, H, D, B = 24, 8, 4.0, 0.2          # cameras shifted by whole pixels (s = 5)
S = int(round(F * B / D))


def _load_maps(mvs, ctx, maps, n_views):
    """Put given plane maps into the context (initial state, no phases)."""
    for v, pl in maps.items():
        hh, ww = pl.shape[:2]
        p = mvs.PMParams(win_radius=5.0, win_samples=6, iters=0, phase_begin=0, phase_end=0,
                         init_mode=mvs.MVS_INIT_GIVEN)
        srcs = [u for u in range(n_views) if u != v][:4]
        mvs.mvs_patchmatch(ctx.h, v, srcs, p, np.ascontiguousarray(pl, np.float32), np.zeros((hh, ww), np.float32))


def _gpu_fuse(mvs, ctx, order, keep=None):
    n_pix = len(order) * H * W
    pts = np.zeros((n_pix, 4), np.float32)
    src = np.zeros((n_pix, 2), np.int32)
    n = mvs.mvs_fuse(ctx.h, order, pts, src, keep_masks=keep)
    return pts[:n], src[:n]


def test_closed_form_plane_equals_oracle(mvs_lib, oracle_lib):
    import torch
    n = 3
    K = np.tile(np.array([[F, 0, CX], [0, F, CY], [0, 0, 1]], np.float64), (n, 1, 1))
    R = np.tile(np.eye(3), (n, 1, 1))
    t = np.array([[-k * B, 0.0, 0.0] for k in range(n)])
    imgs = [np.full((H, W), 128, np.uint8) for _ in range(n)]
    pl = np.zeros((H, W, 4))
    pl[..., 2], pl[..., 3] = -1.0, D
    maps = {v: pl for v in range(n)}
    ctx = mvs_lib.Context(K, R, t, imgs, stream=torch.cuda.current_stream())
    try:
        _load_maps(mvs_lib, ctx, maps, n)
        pts, src = _gpu_fuse(mvs_lib, ctx, [0, 1, 2])
    finally:
        ctx.close()
    assert len(pts) == H * (W + 2 * S) and pts[:, 3].sum() == 3 * H * W
    opts, osv, osp = oracle_lib.fuse(oracle_lib.Scene(K, R, t, imgs), [0, 1, 2], maps)
    assert np.array_equal(src[:, 0], osv) and np.array_equal(src[:, 1], osp)
    assert _close(pts, opts)


@pytest.fixture(scope="module")
def fused_scene(mvs_lib):
    """Five views of the small synthetic scene: PatchMatch maps and
    geometric-filter masks computed by the library."""
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=128, H=96, n_src=4, seed=13, baseline_frac=0.1)
    n = len(sc.images)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=3, seed=9)
    hh, ww = sc.images[0].shape
    maps = {}
    for v in range(n):
        pl = np.zeros((hh, ww, 4), np.float32)
        co = np.zeros((hh, ww), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, v, [u for u in range(n) if u != v], p, pl, co)
        maps[v] = pl
    keep = {}
    for v in range(n):
        k = np.zeros((hh, ww), np.uint8)
        mvs_lib.mvs_geo_filter(ctx.h, v, [u for u in range(n) if u != v], mvs_lib.FilterParams(), k)
        keep[v] = k
    yield sc, ctx, maps, keep
    ctx.close()


@pytest.mark.parametrize("order", [[0, 1, 2, 3, 4], [4, 2, 0, 3, 1]])
def test_patchmatch_maps_equal_oracle(fused_scene, mvs_lib, oracle_lib, order):
    sc, ctx, maps, keep = fused_scene
    hh, ww = sc.images[0].shape
    cap = len(order) * hh * ww
    pts = np.zeros((cap, 4), np.float32)
    src = np.zeros((cap, 2), np.int32)
    owner = np.zeros(cap, np.int64)
    n = mvs_lib.mvs_fuse(ctx.h, order, pts, src, keep_masks=[keep[v] for v in order], owner=owner)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    fmaps = {v: maps[v].astype(np.float64) for v in order}
    opts, osv, osp, oown, st = oracle_lib.fuse(osc, order, fmaps, keep=keep, hint=owner, band_px=BAND_PX,
                                               band_rel=BAND_REL, stats=True)
    frac = st["fragile"] / st["projections"]
    print(f"fusion: {st['projections']} projections, {st['fragile']} fragile ({frac:.2e}), "
          f"{st['resolved_by_hint']} taken the library's way")
    assert frac < 0.01
    assert n == len(opts)
    assert np.array_equal(src[:n, 0], osv) and np.array_equal(src[:n, 1], osp)
    assert np.array_equal(owner, oown)
    assert _close(pts[:n], opts)
    # with no decision taken the library's way, the oracle on its own gives
    # the same fusion
    if st["resolved_by_hint"] == 0:
        _, _, _, free_own, _ = oracle_lib.fuse(osc, order, fmaps, keep=keep, stats=True)
        assert np.array_equal(free_own, owner)
    # merging happened, and every kept pixel ends in exactly one point
    assert (opts[:, 3] > 1).mean() > 0.3
    assert opts[:, 3].sum() == sum(int(((maps[v][..., 3] > 0) & (keep[v] > 0)).sum()) for v in order)


def test_device_buffers_and_capacity(fused_scene, mvs_lib):
    import torch
    sc, ctx, maps, keep = fused_scene
    hh, ww = sc.images[0].shape
    order = [0, 1, 2, 3, 4]
    cap = 5 * hh * ww
    h_pts = np.zeros((cap, 4), np.float32)
    n = mvs_lib.mvs_fuse(ctx.h, order, h_pts, None, keep_masks=[keep[v] for v in order])
    d_pts = torch.zeros((cap, 4), dtype=torch.float32, device="cuda")
    d_src = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    d_keep = [torch.from_numpy(keep[v]).cuda() for v in order]
    h_own = np.zeros(cap, np.int64)
    mvs_lib.mvs_fuse(ctx.h, order, h_pts, None, keep_masks=[keep[v] for v in order], owner=h_own)
    d_own = torch.zeros(cap, dtype=torch.int64, device="cuda")
    n2 = mvs_lib.mvs_fuse(ctx.h, order, d_pts, d_src, keep_masks=d_keep, owner=d_own)
    torch.cuda.synchronize()
    assert n2 == n and np.array_equal(d_pts.cpu().numpy()[:n], h_pts[:n])
    assert np.array_equal(d_own.cpu().numpy(), h_own)
    # every pixel with depth that is kept belongs to one point, the others to none
    present = np.concatenate([((maps[v][..., 3] > 0) & (keep[v] > 0)).ravel() for v in order])
    assert ((h_own >= 0) == present).all() and h_own.max() == n - 1
    assert np.array_equal(np.bincount(h_own[h_own >= 0], minlength=n), h_pts[:n, 3].astype(np.int64))
    # too small a buffer: the call fails and writes the first points only
    small = np.zeros((n - 7, 4), np.float32)
    with pytest.raises(mvs_lib.MvsError):
        mvs_lib.mvs_fuse(ctx.h, order, small, None, keep_masks=[keep[v] for v in order])
    assert np.array_equal(small, h_pts[: n - 7])


def test_single_view_and_empty_masks(fused_scene, mvs_lib, oracle_lib):
    sc, ctx, maps, keep = fused_scene
    hh, ww = sc.images[0].shape
    # one view: every kept pixel is its own point
    pts = np.zeros((hh * ww, 4), np.float32)
    src = np.zeros((hh * ww, 2), np.int32)
    n = mvs_lib.mvs_fuse(ctx.h, [3], pts, src, keep_masks=[keep[3]])
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    opts, osv, osp = oracle_lib.fuse(osc, [3], {3: maps[3].astype(np.float64)}, keep={3: keep[3]})
    assert n == len(opts) == int(((maps[3][..., 3] > 0) & (keep[3] > 0)).sum())
    assert _close(pts[:n], opts) and (pts[:n, 3] == 1).all() and np.array_equal(src[:n, 1], osp)
    # nothing kept: no points
    zero = np.zeros((hh, ww), np.uint8)
    assert mvs_lib.mvs_fuse(ctx.h, [0, 1], pts, None, keep_masks=[zero, zero]) == 0
