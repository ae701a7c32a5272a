"""Synthetic hypothesis sets for the plane-hypothesis selection tests (input
generation only; no step of the method is computed here)."""
import numpy as np


def slanted_hole_case(rng, W=36, H=28):
    """Slanted plane with a hole; per hole pixel four hypotheses, of which
    one (a random direction) is the exact planar depth at the lowest cost and
    the others perturbed depths at higher costs; some invalid, some ties."""
    from paper_2104_06165_gb300 import scenes
    n_true = np.array([0.25, -0.3, -1.0])
    n_true /= np.linalg.norm(n_true)
    sc = scenes.make_plane_scene(W=W, H=H, n_src=1, seed=3, depth=5.0, normal=n_true)
    gt = sc.gt_depth
    known = np.ones((H, W), np.uint8)
    known[6:22, 8:28] = 0
    hyp = gt[..., None] * (1.0 + rng.uniform(0.02, 0.1, (H, W, 4)) * rng.choice([-1, 1], (H, W, 4)))
    hcost = rng.uniform(0.3, 1.9, (H, W, 4))
    valid = (rng.random((H, W, 4)) < 0.8).astype(np.uint8)
    best = rng.integers(0, 4, (H, W))
    yy, xx = np.mgrid[0:H, 0:W]
    hyp[yy, xx, best] = gt
    hcost[yy, xx, best] = rng.uniform(0.0, 0.25, (H, W))
    valid[yy, xx, best] = 1
    # ties: a perturbed hypothesis at a higher index with the same cost never wins
    tie = (rng.random((H, W)) < 0.3) & (best < 3)
    hcost[yy[tie], xx[tie], 3] = hcost[yy[tie], xx[tie], best[tie]]
    valid[yy[tie], xx[tie], 3] = 1
    plane = np.concatenate([sc.gt_normal, gt[..., None]], -1) * known[..., None]
    return sc, n_true, known, hyp, valid, hcost, plane, best
