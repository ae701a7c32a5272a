"""Pins of the FP64 proposal-network oracle (oracle/cnn_oracle.py) against
what mathematics fixes independently of its own code: a library correlation,
adjointness of every linear layer, central finite differences of the loss,
closed forms of the loss and of the first Adam step, and torch's bfloat16
conversion."""
import numpy as np
import pytest

from oracle import cnn_oracle as cn


def _theta(rng, scale=1.0):
    layers = []
    for i, (ci, co, t) in enumerate(cn.LAYERS):
        sd = scale * np.sqrt(2.0 / (t * ci)) * (0.1 if i == cn.HEAD else 1.0)
        layers.append((rng.normal(0, sd, (co, t, ci)), rng.normal(0, 0.05, co)))
    return cn.pack(layers)


def _state(rng, H, W):
    img = rng.integers(20, 236, (H, W)).astype(np.uint8)
    n = rng.normal(0, 1, (H, W, 3))
    n[..., 2] = -np.abs(n[..., 2]) - 1.0
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    plane = np.concatenate([n, rng.uniform(2.0, 8.0, (H, W, 1))], -1)
    cost = rng.uniform(0, 2, (H, W))
    return img, plane, cost


def test_conv_is_the_library_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.normal(size=(7, 9, 3))
    w = rng.normal(size=(2, 9, 3))
    b = rng.normal(size=2)
    out = cn.conv(x, w, b)
    for o in range(2):
        ref = b[o] + sum(signal.correlate2d(x[..., i], w[o, :, i].reshape(3, 3), mode="same")
                         for i in range(3))
        assert np.allclose(out[..., o], ref, atol=1e-12)
    w1 = rng.normal(size=(4, 1, 3))
    assert np.allclose(cn.conv(x, w1, np.zeros(4)), np.einsum("hwi,oi->hwo", x, w1[:, 0]), atol=1e-12)


def test_linear_layers_and_their_backward_are_adjoint():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(8, 6, 5))
    g = rng.normal(size=(4, 3, 5))
    assert np.isclose(np.vdot(cn.pool(x), g), np.vdot(x, cn.pool_backward(g)))
    xs = rng.normal(size=(4, 3, 5))
    gs = rng.normal(size=(8, 6, 5))
    assert np.isclose(np.vdot(cn.up(xs), gs), np.vdot(xs, cn.up_backward(gs)))
    for taps in (9, 1):
        w = rng.normal(size=(7, taps, 5))
        gout = rng.normal(size=(8, 6, 7))
        gx, gw, gb = cn.conv_backward(x, w, gout)
        zero = np.zeros(7)
        assert np.isclose(np.vdot(cn.conv(x, w, zero), gout), np.vdot(x, gx))      # adjoint in x
        assert np.isclose(np.vdot(cn.conv(x, w, zero), gout), np.vdot(w, gw))      # linear in w
        assert np.allclose(gb, gout.sum(axis=(0, 1)))


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    H, W = 32, 32
    img, plane, cost = _state(rng, H, W)
    img2, target, _ = _state(rng, H, W)
    mask = (rng.uniform(size=(H, W)) < 0.7).astype(np.uint8)
    theta = _theta(rng)
    f = lambda th: cn.loss_and_grad(th, img, plane, cost, target, mask, 2.0, 8.0)[0]
    _, g, _ = cn.loss_and_grad(theta, img, plane, cost, target, mask, 2.0, 8.0)
    # sample parameters of every layer, weights and biases
    idx, off = [], 0
    for ci, co, t in cn.LAYERS:
        nw = co * t * ci
        idx += list(rng.choice(nw, 4, replace=False) + off) + list(rng.choice(co, 2, replace=False) + off + nw)
        off += nw + co
    eps = 1e-6
    bad = 0
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (f(tp) - f(tm)) / (2 * eps)
        if not abs(fd - g[i]) <= 1e-7 + 1e-4 * abs(g[i]):
            bad += 1
    assert bad <= 1, bad        # one sample may straddle a ReLU / |.| / argmin kink


def test_loss_closed_forms():
    d_lo, d_hi = 2.0, 8.0
    span = 1 / d_lo - 1 / d_hi
    nt = np.array([0.2, -0.1, -1.0])
    nt /= np.linalg.norm(nt)
    target = np.zeros((1, 1, 4))
    target[0, 0] = [*nt, 4.0]
    mask = np.ones((1, 1), np.uint8)

    def logit(p):
        return np.log(p / (1 - p))

    # proposal 2 equal to the target -> loss 0 whatever the others are
    y = np.random.default_rng(4).normal(size=(1, 1, 16))
    y[0, 0, 8] = logit((1 / 4.0 - 1 / d_hi) / span)
    y[0, 0, 9:12] = 3.7 * nt
    total, g = cn.loss(y, target, mask, d_lo, d_hi)
    assert abs(total) < 1e-12
    # single proposal off by 0.1 of the inverse-depth span and tilted by alpha
    alpha = 0.3
    axis = np.cross(nt, [1.0, 0, 0])
    axis /= np.linalg.norm(axis)
    n1 = np.cos(alpha) * nt + np.sin(alpha) * np.cross(axis, nt)
    y = np.zeros((1, 1, 16))
    y[0, 0, 0::4] = 20.0           # other proposals far (rho at 1/d_lo)
    y[0, 0, 1::4] = 1.0
    y[0, 0, 0] = logit((1 / 4.0 + 0.1 * span - 1 / d_hi) / span)
    y[0, 0, 1:4] = 0.5 * n1
    total, _ = cn.loss(y, target, mask, d_lo, d_hi)
    assert np.isclose(total, 0.1 + cn.LAMBDA_N * (1 - np.cos(alpha)), atol=1e-12)
    # pixels without a target add nothing
    total, g = cn.loss(y, target, np.zeros((1, 1), np.uint8), d_lo, d_hi)
    assert total == 0 and not g.any()


def test_proposals_face_the_camera_inside_the_depth_range():
    rng = np.random.default_rng(5)
    y = rng.normal(0, 3, (16, 16, 16))
    Kinv = np.linalg.inv(np.array([[300.0, 0, 8], [0, 300.0, 8], [0, 0, 1]]))
    pr = cn.propose(y, Kinv, 2.0, 8.0)
    assert pr.shape == (16, 16, 4, 4)
    assert np.allclose(np.linalg.norm(pr[..., :3], axis=-1), 1.0)
    assert (pr[..., 3] >= 2.0 - 1e-12).all() and (pr[..., 3] <= 8.0 + 1e-12).all()
    xs, ys = np.meshgrid(np.arange(16.0), np.arange(16.0))
    ray = np.stack([xs, ys, np.ones_like(xs)], -1) @ Kinv.T
    assert (np.einsum("hwkc,hwc->hwk", pr[..., :3], ray) <= 0).all()


def test_first_adam_step_is_lr_times_sign():
    rng = np.random.default_rng(6)
    th = rng.normal(size=100)
    g = rng.normal(size=100)
    new, m, v = cn.adam(th, g, np.zeros(100), np.zeros(100), 1, 1e-3)
    assert np.allclose(new, th - 1e-3 * np.sign(g), atol=1e-10)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    assert cn.to_bf16(1.0 + 2.0 ** -8) == 1.0                 # tie -> even
    assert cn.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (up)
    rng = np.random.default_rng(7)
    a = rng.normal(0, 10, 10000).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cn.to_bf16(a), ref)


def test_parameter_count_and_layout():
    assert cn.n_params() == sum(co * t * ci + co for ci, co, t in cn.LAYERS)
    rng = np.random.default_rng(8)
    th = rng.normal(size=cn.n_params())
    assert np.array_equal(cn.pack(cn.unpack(th)), th)
    # decoder inputs are up-sampled channels + the encoder skip of the level
    for lv in (3, 2, 1, 0):
        below = cn.LAYERS[cn.E[4]][1] if lv == 3 else cn.LAYERS[cn.D[lv + 1]][1]
        assert cn.LAYERS[cn.D[lv]][0] == below + cn.LAYERS[cn.E[lv]][1]
