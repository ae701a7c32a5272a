"""Learned plane proposals: training driver and the learned PatchMatch flow.

The network (declared in include/mvs.h, kernels in csrc/cnn_kernels.cu) has
no counterpart in the paper.  It sees a reference image with the PatchMatch
state after one iteration and proposes K = 4 planes per pixel; the remaining
iterations score those planes as extra propagation candidates with the
Eq. 5 cost, which still decides.

Training data are depth maps the plain pipeline produces on seeded synthetic
scenes (no ground truth is used for training): input = state after one
iteration, target = the plain 8-iteration map on pixels whose final cost is
below ``TARGET_COST``.  Every step runs in the library's kernels (forward,
loss, backward, Adam); this module only schedules calls and slices crops.

    python -m paper_2104_06165_gb300.proposals --out weights.npy
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from . import mvs, scenes

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "proposal_unet.npy")
K_PROP = 4
TARGET_COST = 0.5
# scenes of the learned-proposal workload: the high-resolution generator at
# 1536 x 1024, 10 sources at 15..40 deg, blank patches on the quads and on
# the background covering about half of the reference image
SCENE = dict(W=1536, H=1024, n_src=10, flat_frac=0.5, flat_bg=0.5)
TRAIN_SEEDS = range(0, 200)
EVAL_SEEDS = range(1000, 1004)


def scene(seed, W=SCENE["W"], H=SCENE["H"], n_src=SCENE["n_src"]):
    angles = list(np.linspace(15.0, 40.0, n_src))
    return scenes.make_scene(W=W, H=H, n_src=n_src, seed=seed, view_angles=angles, n_textured=4, n_flat=4,
                             flat_frac=SCENE["flat_frac"], flat_bg=SCENE["flat_bg"])


def pm_params(seed, iters=8, **kw):
    """Window of the high-resolution workload: 21 x 21 at dilation 2."""
    return mvs.PMParams(win_radius=10.0, win_samples=11, sigma_s=5.0, sigma_c=0.2, d_lo=2.0, d_hi=8.0,
                        iters=iters, seed=seed, **kw)


def cnn_flops(W, H):
    """Algorithmic flops of one forward pass (2 per multiply-add of every
    convolution) at a W x H input."""
    levels = [0, 1, 2, 3, 4, 3, 2, 1, 0, 0]
    layers = [(16, 32, 9), (32, 48, 9), (48, 64, 9), (64, 96, 9), (96, 128, 9),
              (224, 96, 9), (160, 64, 9), (112, 48, 9), (80, 32, 9), (32, 16, 1)]
    return sum(2 * (W >> l) * (H >> l) * co * t * ci for l, (ci, co, t) in zip(levels, layers))


def load_weights(net, path=WEIGHTS):
    mvs.mvs_cnn_set_params(net, np.load(path))


def learned_patchmatch(ctx, ref, srcs, params, net, plane, cost, proposals, iters=4, first=1):
    """Random initialisation and ``first`` plain iterations, proposals from
    the network on that state, then iterations first..iters-1 with the
    proposals as extra propagation candidates.  plane / cost / proposals:
    device tensors (H, W, 4), (H, W), (H, W, 4, 4)."""
    p0 = mvs.PMParams(**{**params.__dict__, "iters": iters, "phase_begin": 0, "phase_end": 2 * first,
                         "init_mode": mvs.MVS_INIT_RANDOM, "n_prop": 0, "proposals": None})
    mvs.mvs_patchmatch(ctx.h, ref, srcs, p0, plane, cost)
    mvs.mvs_propose(ctx.h, ref, net, proposals)
    p1 = mvs.PMParams(**{**params.__dict__, "iters": iters, "phase_begin": 2 * first, "phase_end": 2 * iters,
                         "init_mode": mvs.MVS_INIT_GIVEN, "n_prop": K_PROP, "proposals": proposals})
    mvs.mvs_patchmatch(ctx.h, ref, srcs, p1, plane, cost)


def make_example(seed, torch, stream):
    """(img, plane after 1 iteration, its cost, target plane map, mask) on
    the device for one training scene."""
    sc = scene(seed)
    H, W = sc.images[0].shape
    srcs = list(range(1, len(sc.images)))
    dev = "cuda"
    with mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream) as ctx:
        plane = torch.zeros((H, W, 4), dtype=torch.float32, device=dev)
        cost = torch.zeros((H, W), dtype=torch.float32, device=dev)
        p = pm_params(seed, iters=8, phase_end=2)
        mvs.mvs_patchmatch(ctx.h, 0, srcs, p, plane, cost)
        x_plane, x_cost = plane.clone(), cost.clone()
        p = pm_params(seed, iters=8, phase_begin=2, init_mode=mvs.MVS_INIT_GIVEN)
        mvs.mvs_patchmatch(ctx.h, 0, srcs, p, plane, cost)
    img = torch.from_numpy(np.ascontiguousarray(sc.images[0])).to(dev)
    mask = ((cost < TARGET_COST) & (plane[..., 3] > 0)).to(torch.uint8)
    return img, x_plane, x_cost, plane, mask


def train(out=WEIGHTS, steps=3000, crop=(512, 384), lr=1e-3, seed=0, seeds=TRAIN_SEEDS, log=print):
    import torch
    torch.cuda.init()
    stream = torch.cuda.current_stream()
    t0 = time.time()
    data = [make_example(s, torch, stream) for s in seeds]
    torch.cuda.synchronize()
    log(f"data: {len(data)} scenes in {time.time() - t0:.1f} s")
    cw, ch = crop
    net = mvs.mvs_cnn_create(cw, ch, 2.0, 8.0, seed, stream)
    rng = np.random.default_rng(seed)
    t0 = time.time()
    losses = []
    try:
        for it in range(steps):
            img, xp, xc, tp, m = data[rng.integers(len(data))]
            H, W = img.shape
            y0 = int(rng.integers(0, H - ch + 1))
            x0 = int(rng.integers(0, W - cw + 1))
            sl = (slice(y0, y0 + ch), slice(x0, x0 + cw))
            c = [a[sl].contiguous() for a in (img, xp, xc, tp, m)]
            rate = lr * 0.5 * (1 + np.cos(np.pi * it / steps))      # cosine schedule
            loss = mvs.mvs_cnn_backward(net, *c)
            mvs.mvs_cnn_adam_step(net, rate)
            losses.append(loss)
            if (it + 1) % 250 == 0:
                log(f"step {it + 1}: loss {np.mean(losses[-250:]):.4f}  ({time.time() - t0:.1f} s)")
        theta = mvs.mvs_cnn_get_params(net)
    finally:
        mvs.mvs_cnn_destroy(net)
    if out:
        os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
        np.save(out, theta.astype(np.float32))
    return theta, losses


def completeness(plane, gt_depth, tol=0.01):
    """Fraction of all pixels whose depth is within tol (relative) of the
    ground truth."""
    d = plane[..., 3]
    return float((np.abs(d - gt_depth) <= tol * gt_depth).mean())


def evaluate(weights=WEIGHTS, seeds=EVAL_SEEDS, log=print):
    """Completeness and depth-map time of plain 4 / plain 8 / learned 4 on
    held-out scenes."""
    import torch
    stream = torch.cuda.current_stream()
    W, H = SCENE["W"], SCENE["H"]
    net = mvs.mvs_cnn_create(W, H, 2.0, 8.0, 0, stream)
    rows = []
    try:
        mvs.mvs_cnn_set_params(net, np.load(weights) if isinstance(weights, str) else weights)
        for s in seeds:
            sc = scene(s)
            srcs = list(range(1, len(sc.images)))
            with mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream) as ctx:
                plane = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
                cost = torch.zeros((H, W), dtype=torch.float32, device="cuda")
                props = torch.zeros((H, W, K_PROP, 4), dtype=torch.float32, device="cuda")
                res = {}
                for name in ("plain4", "plain8", "learned4"):
                    for rep in range(2):          # the first run warms up
                        torch.cuda.synchronize()
                        t = time.perf_counter()
                        if name == "learned4":
                            learned_patchmatch(ctx, 0, srcs, pm_params(s), net, plane, cost, props, iters=4)
                        else:
                            mvs.mvs_patchmatch(ctx.h, 0, srcs, pm_params(s, iters=int(name[5:])), plane, cost)
                        torch.cuda.synchronize()
                        ms = (time.perf_counter() - t) * 1e3
                    res[name] = (completeness(plane.cpu().numpy(), sc.gt_depth), ms)
            rows.append(res)
            log(f"seed {s}: " + "  ".join(f"{k} {v[0]:.4f} ({v[1]:.1f} ms)" for k, v in res.items()))
    finally:
        mvs.mvs_cnn_destroy(net)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--scenes", type=int, default=len(TRAIN_SEEDS))
    ap.add_argument("--eval-only", action="store_true")
    args = ap.parse_args()
    if not args.eval_only:
        train(args.out, steps=args.steps, lr=args.lr, seeds=range(args.scenes))
    evaluate(args.out)


if __name__ == "__main__":
    main()
