"""Parity at the full size of the measured workload (3072 x 2048 reference,
10 sources, 21 x 21 window at dilation 2, 8 iterations), in the launch
configuration bench.py times: properties of every pixel, and the oracle's
cost of the GPU's final plane at sampled pixels."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

COST_TOL = 1e-4
MARGIN = 1e-3


def test_full_size_depth_map(mvs_lib, oracle_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.scene_highres(seed=0)
    H, W = sc.images[0].shape
    assert (W, H) == (3072, 2048)
    srcs = list(range(1, 11))
    p = mvs_lib.PMParams(win_radius=10.0, win_samples=11, sigma_s=5.0, sigma_c=0.2, d_lo=2.0, d_hi=8.0, iters=8,
                         seed=1)
    with mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream()) as ctx:
        plane = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        cost = torch.empty((H, W), dtype=torch.float32, device="cuda")
        mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, p, plane, cost)
        pl = plane.cpu().numpy()
        co = cost.cpu().numpy()
    # every pixel: a valid plane facing the camera inside the depth range,
    # a cost in [1e-6, C_max]
    d = pl[..., 3]
    assert ((d >= 2.0) & (d <= 8.0)).all()
    assert np.abs(np.linalg.norm(pl[..., :3], axis=-1) - 1).max() < 1e-5
    xs, ys = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ray = np.stack([xs, ys, np.ones_like(xs)], -1) @ np.linalg.inv(sc.K[0]).T
    assert (np.einsum("hwc,hwc->hw", pl[..., :3].astype(np.float64), ray) < 0).all()
    assert ((co >= 1e-6 * 0.999) & (co <= 2.0)).all()
    # sampled pixels: the oracle's cost of the GPU's plane equals the GPU's cost
    rng = np.random.default_rng(0)
    sx = rng.integers(0, W, 60)
    sy = rng.integers(0, H, 60)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    oc, mg = oracle_lib.cost_at(osc, 0, srcs, p, sx, sy, pl[sy, sx].astype(np.float64))
    firm = mg > MARGIN
    assert firm.mean() > 0.9
    err = np.abs(co[sy, sx] - oc)[firm]
    assert err.max() <= COST_TOL, err.max()
    # the map is a depth map of the scene: most textured pixels within 1 %
    tex = sc.gt_textured
    ok = np.abs(d - sc.gt_depth) <= 0.01 * sc.gt_depth
    assert ok[tex].mean() > 0.95
