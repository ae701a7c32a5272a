"""GPU-vs-oracle parity of the learned plane-proposal network and of the
proposal stage of PatchMatch (through the C ABI).

Tolerances.  The library stores the input, weights, activations and
activation gradients in bfloat16 and sums in fp32; the oracle's bf16 mode
rounds at the same points and sums in fp64.  The two differ only where the
fp32 summation error (a few 1e-6 relative for sums of up to 2016 products)
moves a value across a bf16 rounding boundary; such a value then differs by
one bf16 step (2^-8 relative) and the difference spreads through the later
layers.  How far it spreads is a property of the network and its weights,
so each test measures it: the oracle is run a second time with the weights
perturbed by 2e-6 relative (the size of the fp32 summation error), and the
GPU must stay within 4x that self-disagreement of the bf16 oracle (plus a
floor of 1e-4).  On GB300 the GPU's head output sat at 1.3e-3 relative L2
and its weight gradients at up to 1.0e-2 per layer.  Against the exact fp64
network (no rounding) the gradient directions agree to cosine > 0.99.
"""
import copy

import numpy as np
import pytest

from oracle import cnn_oracle as cn

pytestmark = pytest.mark.gpu

W, H = 64, 48
D_LO, D_HI = 2.0, 8.0


def _state(rng):
    img = rng.integers(20, 236, (H, W)).astype(np.uint8)
    n = rng.normal(0, 1, (H, W, 3))
    n[..., 2] = -np.abs(n[..., 2]) - 1.0
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    plane = np.concatenate([n, rng.uniform(D_LO, D_HI, (H, W, 1))], -1).astype(np.float32)
    cost = rng.uniform(0, 2, (H, W)).astype(np.float32)
    return img, plane, cost


def _dev(torch, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.fixture(scope="module")
def case(mvs_lib):
    import torch
    rng = np.random.default_rng(21)
    img, plane, cost = _state(rng)
    _, target, _ = _state(rng)
    mask = (rng.uniform(size=(H, W)) < 0.7).astype(np.uint8)
    net = mvs_lib.mvs_cnn_create(W, H, D_LO, D_HI, 99, torch.cuda.current_stream())
    # biases of a trained network are not zero: give them a spread
    theta = mvs_lib.mvs_cnn_get_params(net).astype(np.float64)
    off = 0
    for ci, co, t in cn.LAYERS:
        off += co * t * ci
        theta[off: off + co] = rng.normal(0, 0.05, co)
        off += co
    mvs_lib.mvs_cnn_set_params(net, theta.astype(np.float32))
    theta = mvs_lib.mvs_cnn_get_params(net).astype(np.float64)
    yield dict(net=net, theta=theta, img=img, plane=plane, cost=cost, target=target, mask=mask)
    mvs_lib.mvs_cnn_destroy(net)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _perturbed(theta, seed=0, eps=2e-6):
    rng = np.random.default_rng(seed)
    return theta * (1 + eps * rng.standard_normal(theta.shape))


def _layer_slices():
    off = 0
    for ci, co, t in cn.LAYERS:
        n = co * t * ci + co
        yield slice(off, off + n)
        off += n


def test_forward_matches_oracle(case, mvs_lib):
    import torch
    d_img, d_pl, d_co = _dev(torch, case["img"], case["plane"], case["cost"])
    out = torch.zeros((H, W, 16), dtype=torch.float32, device="cuda")
    mvs_lib.mvs_cnn_forward(case["net"], d_img, d_pl, d_co, out)
    y = out.cpu().numpy().astype(np.float64)
    x = cn.make_input(case["img"], case["plane"].astype(np.float64), case["cost"].astype(np.float64), D_LO, D_HI)
    y_bf, _ = cn.forward(case["theta"], x, bf16=True)
    y_pt, _ = cn.forward(_perturbed(case["theta"]), x, bf16=True)
    y_ex, _ = cn.forward(case["theta"], x, bf16=False)
    noise = _rel(y_pt, y_bf)
    assert _rel(y, y_bf) <= 4 * noise + 1e-4, (_rel(y, y_bf), noise)
    assert _rel(y, y_ex) <= 3e-2          # bf16 storage against the exact network


def test_gradients_match_oracle(case, mvs_lib):
    import torch
    d = _dev(torch, case["img"], case["plane"], case["cost"], case["target"], case["mask"])
    loss = mvs_lib.mvs_cnn_backward(case["net"], *d)
    g = mvs_lib.mvs_cnn_get_grads(case["net"]).astype(np.float64)
    pl64 = case["plane"].astype(np.float64)
    args = (case["img"], pl64, case["cost"].astype(np.float64), case["target"].astype(np.float64), case["mask"],
            D_LO, D_HI)
    L_bf, g_bf, _ = cn.loss_and_grad(case["theta"], *args, bf16=True)
    _, g_pt, _ = cn.loss_and_grad(_perturbed(case["theta"]), *args, bf16=True)
    _, g_ex, _ = cn.loss_and_grad(case["theta"], *args, bf16=False)
    assert abs(loss - L_bf) <= 1e-3 * abs(L_bf)
    for i, sl in enumerate(_layer_slices()):
        a, b, e = g[sl], g_bf[sl], g_ex[sl]
        noise = _rel(g_pt[sl], b)
        assert _rel(a, b) <= 4 * noise + 1e-4, f"layer {i}: relative error {_rel(a, b):.3g} (noise {noise:.3g})"
        cos = a @ e / (np.linalg.norm(a) * np.linalg.norm(e))
        assert cos > 0.99, f"layer {i}: cosine to the exact gradient {cos:.4f}"


def test_adam_step_matches_oracle(mvs_lib):
    import torch
    rng = np.random.default_rng(5)
    img, plane, cost = _state(rng)
    _, target, _ = _state(rng)
    mask = np.ones((H, W), np.uint8)
    net = mvs_lib.mvs_cnn_create(W, H, D_LO, D_HI, 7, torch.cuda.current_stream())
    try:
        d = _dev(torch, img, plane, cost, target, mask)
        th, m, v = mvs_lib.mvs_cnn_get_params(net).astype(np.float64), 0.0, 0.0
        for t in (1, 2, 3):
            mvs_lib.mvs_cnn_backward(net, *d)
            g = mvs_lib.mvs_cnn_get_grads(net).astype(np.float64)
            mvs_lib.mvs_cnn_adam_step(net, 1e-3)
            th, m, v = cn.adam(th, g, m, v, t, 1e-3)
            got = mvs_lib.mvs_cnn_get_params(net).astype(np.float64)
            assert np.abs(got - th).max() <= 1e-6, np.abs(got - th).max()
            th = got
    finally:
        mvs_lib.mvs_cnn_destroy(net)


def test_decode_matches_oracle(case, mvs_lib):
    """Proposals decoded on the GPU from its own head output equal the
    oracle's decoding of that output."""
    import torch
    d_img, d_pl, d_co = _dev(torch, case["img"], case["plane"], case["cost"])
    out = torch.zeros((H, W, 16), dtype=torch.float32, device="cuda")
    mvs_lib.mvs_cnn_forward(case["net"], d_img, d_pl, d_co, out)
    props = torch.zeros((H, W, 4, 4), dtype=torch.float32, device="cuda")
    Kinv = np.linalg.inv(np.array([[60.0, 0, 31.5], [0, 60.0, 23.5], [0, 0, 1]]))
    mvs_lib.mvs_cnn_propose(case["net"], d_img, d_pl, d_co, Kinv, props)
    got = props.cpu().numpy().astype(np.float64)
    want = cn.propose(out.cpu().numpy().astype(np.float64), Kinv, D_LO, D_HI)
    assert np.abs(got[..., 3] - want[..., 3]).max() <= 1e-5 * D_HI
    assert np.abs(got[..., :3] - want[..., :3]).max() <= 1e-5


def test_training_lowers_the_loss(mvs_lib):
    import torch
    rng = np.random.default_rng(8)
    img, plane, cost = _state(rng)
    # a smooth target the network can fit: the input planes blurred to one
    # plane per 16 x 16 block
    target = plane.copy()
    for y in range(0, H, 16):
        for x in range(0, W, 16):
            target[y:y + 16, x:x + 16] = plane[y + 8, x + 8]
    mask = np.ones((H, W), np.uint8)
    net = mvs_lib.mvs_cnn_create(W, H, D_LO, D_HI, 3, torch.cuda.current_stream())
    try:
        d = _dev(torch, img, plane, cost, target, mask)
        losses = []
        for it in range(150):
            losses.append(mvs_lib.mvs_cnn_backward(net, *d))
            mvs_lib.mvs_cnn_adam_step(net, 2e-3)
        assert np.mean(losses[-10:]) < 0.6 * np.mean(losses[:10]), (losses[:10], losses[-10:])
    finally:
        mvs_lib.mvs_cnn_destroy(net)


def test_shape_and_argument_checks(mvs_lib):
    import torch
    net = mvs_lib.mvs_cnn_create(64, 48, D_LO, D_HI, 0, torch.cuda.current_stream())
    try:
        img = torch.zeros((40, 40), dtype=torch.uint8, device="cuda")     # not a multiple of 16
        pl = torch.zeros((40, 40, 4), dtype=torch.float32, device="cuda")
        co = torch.zeros((40, 40), dtype=torch.float32, device="cuda")
        out = torch.zeros((40, 40, 16), dtype=torch.float32, device="cuda")
        with pytest.raises(mvs_lib.MvsError) as e:
            mvs_lib.mvs_cnn_forward(net, img, pl, co, out)
        assert e.value.status == mvs_lib.MVS_EINVAL
        with pytest.raises(ValueError):
            mvs_lib.mvs_cnn_forward(net, img.cpu(), pl, co, out)
    finally:
        mvs_lib.mvs_cnn_destroy(net)
    with pytest.raises(mvs_lib.MvsError):
        mvs_lib.mvs_cnn_create(60, 48, D_LO, D_HI, 0, None)


# --------------------------------------------------------------------------
# proposals inside PatchMatch
# --------------------------------------------------------------------------
COST_TOL = 1e-4
TIE_BAND = 2e-4
MARGIN = 1e-3


@pytest.fixture(scope="module")
def small(mvs_lib, oracle_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=4, seed=17, baseline_frac=0.1)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, sigma_s=5.0, sigma_c=0.2, iters=3, seed=4321)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    yield sc, p, ctx, osc, [1, 2, 3, 4]
    ctx.close()


def _proposals(sc, rng, k=4):
    """Seeded proposals: the true plane with depth noise, a random
    fronto-parallel plane, the true normal at a random depth, and a slot
    outside the depth range."""
    Hh, Ww = sc.gt_depth.shape
    gt_d = np.where(sc.gt_depth > 0, sc.gt_depth, 5.0)
    pr = np.zeros((Hh, Ww, k, 4), np.float32)
    pr[..., 0, :3] = sc.gt_normal
    pr[..., 0, 3] = gt_d * (1 + rng.normal(0, 0.003, (Hh, Ww)))
    pr[..., 1, :3] = [0.0, 0.0, -1.0]
    pr[..., 1, 3] = rng.uniform(D_LO, D_HI, (Hh, Ww))
    pr[..., 2, :3] = sc.gt_normal
    pr[..., 2, 3] = rng.uniform(D_LO, D_HI, (Hh, Ww))
    pr[..., 3, :3] = [0.0, 0.0, -1.0]
    pr[..., 3, 3] = 9.0
    return pr


def test_phase_with_proposals_lockstep(small, mvs_lib, oracle_lib):
    import torch
    sc, p, ctx, osc, srcs = small
    rng = np.random.default_rng(2)
    props = _proposals(sc, rng)
    d_props = torch.from_numpy(props).cuda()
    q0 = copy.copy(p)
    q0.iters, q0.phase_begin, q0.phase_end = 0, 0, 0
    Hh, Ww = sc.gt_depth.shape
    pl = np.zeros((Hh, Ww, 4), np.float32)
    co = np.zeros((Hh, Ww), np.float32)
    mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q0, pl, co)
    yy, xx = np.mgrid[0:Hh, 0:Ww]
    took = 0
    for ph in range(4):
        q = copy.copy(p)
        q.phase_begin, q.phase_end, q.init_mode = ph, ph + 1, mvs_lib.MVS_INIT_GIVEN
        q.n_prop, q.proposals = 4, d_props
        g_pl, g_co = pl.copy(), co.copy()
        mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q, g_pl, g_co)
        o_pl, o_co, diag = oracle_lib.phase(osc, 0, srcs, p, ph, pl.astype(np.float64), co.astype(np.float64),
                                            proposals=props.astype(np.float64))
        other = ((xx + yy) & 1) != (ph & 1)
        assert np.array_equal(g_pl[other], pl[other]) and np.array_equal(g_co[other], co[other])
        same = (np.abs(g_pl[..., 3] - o_pl[..., 3]) <= 1e-4 * o_pl[..., 3]) & \
               (np.abs(g_pl[..., :3] - o_pl[..., :3]).max(-1) <= 1e-3)
        tie = (diag["gap_prop"] < TIE_BAND) | (diag["gap_ref"] < TIE_BAND) | (diag["margin"] < MARGIN)
        active = ~other
        unexplained = active & ~same & ~tie
        assert unexplained.sum() <= max(2, int(0.0005 * active.sum())), \
            f"phase {ph}: {unexplained.sum()} unexplained decision flips"
        agree = active & same & (diag["margin"] >= MARGIN)
        assert np.abs(g_co - o_co)[agree].max() <= COST_TOL
        took += (active & (diag["win_prop"] >= 8)).sum()
        pl, co = g_pl, g_co
    assert took > 0.05 * Hh * Ww       # the proposals were in play


def test_proposal_arguments_are_checked(small, mvs_lib):
    import torch
    sc, p, ctx, osc, srcs = small
    Hh, Ww = sc.gt_depth.shape
    pl = np.zeros((Hh, Ww, 4), np.float32)
    co = np.zeros((Hh, Ww), np.float32)
    for n_prop, props in ((4, None), (9, torch.zeros((Hh, Ww, 9, 4), device="cuda"))):
        q = copy.copy(p)
        q.n_prop, q.proposals = n_prop, props
        with pytest.raises(mvs_lib.MvsError) as e:
            mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q, pl, co)
        assert e.value.status == mvs_lib.MVS_EINVAL


# --------------------------------------------------------------------------
# what the trained network gains (held-out scene of the learned workload)
# --------------------------------------------------------------------------
def test_trained_proposals_gain(mvs_lib):
    """Learned proposals (1 plain iteration, the network, 3 iterations with
    K = 4 proposals) against plain PatchMatch with 8 and with 4 iterations on
    a held-out 1536 x 1024 scene of the training distribution, scored by
    completeness (depth within 1 % of the ground truth).

    Measured on GB300: learned-4 reaches plain-8's completeness with 78 % of
    its ZNCC evaluations (the phase kernel skips candidates that repeat the
    pixel's plane, which thins plain-8's converged iterations), and equals
    plain-4, which needs fewer evaluations still (these scenes converge in
    two plain iterations, so the proposals find nothing plain PatchMatch
    misses).  The test pins these facts."""
    import torch
    from paper_2104_06165_gb300 import proposals as P
    sc = P.scene(1500)
    Hh, Ww = sc.gt_depth.shape
    srcs = list(range(1, len(sc.images)))
    stream = torch.cuda.current_stream()
    net = mvs_lib.mvs_cnn_create(Ww, Hh, 2.0, 8.0, 0, stream)
    try:
        P.load_weights(net)
        with mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=stream) as ctx:
            plane = torch.zeros((Hh, Ww, 4), dtype=torch.float32, device="cuda")
            cost = torch.zeros((Hh, Ww), dtype=torch.float32, device="cuda")
            props = torch.zeros((Hh, Ww, 4, 4), dtype=torch.float32, device="cuda")
            res = {}
            for name in ("plain4", "plain8", "learned4"):
                mvs_lib.mvs_profile(ctx.h, 1)
                if name == "learned4":
                    P.learned_patchmatch(ctx, 0, srcs, P.pm_params(3), net, plane, cost, props, iters=4)
                else:
                    mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, P.pm_params(3, iters=int(name[5:])), plane, cost)
                evals = mvs_lib.mvs_profile_read(ctx.h)[3]
                mvs_lib.mvs_profile(ctx.h, 0)
                res[name] = (P.completeness(plane.cpu().numpy(), sc.gt_depth), evals)
                if name == "learned4":
                    pr = props.cpu().numpy()
    finally:
        mvs_lib.mvs_cnn_destroy(net)
    (c4, e4), (c8, e8), (cl, el) = res["plain4"], res["plain8"], res["learned4"]
    assert cl >= c8 - 0.002, res            # equal completeness to plain-8 ...
    assert el < e8, res                     # ... with fewer ZNCC evaluations
    assert abs(cl - c4) <= 0.002, res       # no gain over plain-4 ...
    assert el > e4, res                     # ... which evaluates fewer
    # the proposals are planes of the scene: on textured pixels one of the
    # four lies within 1 % of the true depth far more often than chance
    tex = sc.gt_textured
    hit = (np.abs(pr[..., 3] - sc.gt_depth[..., None]) <= 0.01 * sc.gt_depth[..., None]).any(-1)
    assert hit[tex].mean() > 0.5, hit[tex].mean()
