"""Mixed-precision variant (precision = 1): its error against the FP64
oracle, measured and bounded (it is not held to the FP32 path's 1e-4)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_mixed_precision_cost_error_vs_oracle(mvs_lib, oracle_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=4, seed=7, baseline_frac=0.1)
    srcs = [1, 2, 3, 4]
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    try:
        H, W = sc.gt_depth.shape
        gt = np.concatenate([sc.gt_normal, sc.gt_depth[..., None]], -1).astype(np.float32)
        rnd, _ = oracle_lib.init(osc, 0, srcs, mvs_lib.PMParams(win_radius=5.0, win_samples=6, seed=3),
                                 with_cost=False)
        for name, planes in (("gt", gt), ("random", rnd.astype(np.float32))):
            stats = {}
            for prec in (0, 1):
                p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, precision=prec)
                cost = np.zeros((H, W), np.float32)
                mvs_lib.mvs_plane_cost(ctx.h, 0, srcs, p, planes, cost)
                oc, _, mg = oracle_lib.plane_cost(osc, 0, srcs, p, planes.astype(np.float64), with_views=True)
                err = np.abs(cost - oc)[mg > 1e-3]
                stats[prec] = (np.median(err), np.quantile(err, 0.99), err.max())
            print(f"{name}: fp32 median/p99/max {stats[0]}, mixed {stats[1]}")
            med, p99, mx = stats[1]
            assert med < 2e-4 and p99 < 3e-3
    finally:
        ctx.close()


def test_mixed_precision_depth_matches_fp32(mvs_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=192, H=144, n_src=4, seed=9, baseline_frac=0.1)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    try:
        out = {}
        for prec in (0, 1):
            p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=3, seed=5, precision=prec)
            pl = np.zeros((144, 192, 4), np.float32)
            co = np.zeros((144, 192), np.float32)
            mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2, 3, 4], p, pl, co)
            out[prec] = (pl, co)
        gt = sc.gt_depth
        tex = sc.gt_textured
        comp = {k: (np.abs(v[0][..., 3] - gt) / gt < 0.01)[tex].mean() for k, v in out.items()}
        print(f"completeness @1% on textured pixels: fp32 {comp[0]:.4f} mixed {comp[1]:.4f}")
        assert comp[1] > comp[0] - 0.01
    finally:
        ctx.close()
