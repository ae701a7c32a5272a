"""FP64 CPU oracle of the learned plane-proposal network (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; the product path never does.

The network has no counterpart in the paper: it proposes extra plane
hypotheses that the PatchMatch propagation step scores with the Eq. 5 cost.
This module states what the library's network computes, step by step, in
plain numpy (float64):

  input  : 16 channels = image / 255, inverse depth normalised from
           [1/d_hi, 1/d_lo] to [0, 1], normal (3), cost / 2, ten zeros
  encoder: e0 = relu(conv3x3(input)); e_l = relu(conv3x3(avgpool2(e_{l-1})))
           for l = 1..4, with 32, 48, 64, 96, 128 channels
  decoder: d_l = relu(conv3x3(concat(up2(d_{l+1} or e_4), e_l))) for
           l = 3..0, with 96, 64, 48, 32 channels
  head   : y = conv1x1(d_0), 16 channels = 4 x (a, m_x, m_y, m_z)
  decode : rho_k = 1/d_hi + (1/d_lo - 1/d_hi) sigmoid(a_k),
           n_k = m_k / |m_k| turned to face the camera, depth 1 / rho_k
  loss   : L = 1/(W H) sum over target pixels of
           min_k |rho_k - 1/d_t| / (1/d_lo - 1/d_hi) + lambda (1 - |n_k . n_t|)
           (the first k on ties)

Parameters are one flat vector, layer by layer (e0..e4, d3..d0, head), each
as weights [c_out][tap][c_in] (tap = 3 (dy + 1) + (dx + 1)) then bias [c_out].

``bf16=True`` rounds, as the library stores them, the input, the weights
and every stored activation and activation gradient to bfloat16 (round to
nearest even), while sums stay in float64; ``bf16=False`` is the exact
float64 network.  The backward pass is the chain rule written out layer by
layer; its pin is a central finite difference of ``loss`` (tests).
"""
from __future__ import annotations

import numpy as np

# (c_in, c_out, taps) of e0..e4, d3..d0, head
LAYERS = [(16, 32, 9), (32, 48, 9), (48, 64, 9), (64, 96, 9), (96, 128, 9),
          (224, 96, 9), (160, 64, 9), (112, 48, 9), (80, 32, 9), (32, 16, 1)]
E = [0, 1, 2, 3, 4]          # layer index of encoder level l
D = {3: 5, 2: 6, 1: 7, 0: 8}  # layer index of decoder level l
HEAD = 9
K = 4
LAMBDA_N = 0.1


def n_params() -> int:
    return sum(co * t * ci + co for ci, co, t in LAYERS)


def unpack(theta):
    """Flat parameter vector -> list of (w[c_out, tap, c_in], b[c_out])."""
    theta = np.asarray(theta, np.float64)
    out, off = [], 0
    for ci, co, t in LAYERS:
        w = theta[off: off + co * t * ci].reshape(co, t, ci)
        off += co * t * ci
        b = theta[off: off + co]
        off += co
        out.append((w, b))
    assert off == theta.size
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def to_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def make_input(img, plane, cost, d_lo, d_hi):
    """(H, W) uint8 image, (H, W, 4) planes, (H, W) cost -> (H, W, 16)."""
    H, W = img.shape
    rho_lo, rho_hi = 1.0 / d_hi, 1.0 / d_lo
    d = plane[..., 3].astype(np.float64)
    rho = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), rho_lo)
    x = np.zeros((H, W, 16))
    x[..., 0] = img / 255.0
    x[..., 1] = (rho - rho_lo) / (rho_hi - rho_lo)
    x[..., 2:5] = plane[..., :3]
    x[..., 5] = cost * 0.5
    return x


# ---- layers -----------------------------------------------------------
def conv(x, w, b):
    """Zero-padded stride-1 correlation: out[y, x, o] = b[o] +
    sum over taps (dy, dx) and input channels i of
    x[y + dy, x + dx, i] w[o, tap, i]."""
    H, W, _ = x.shape
    taps = w.shape[1]
    out = np.broadcast_to(b, (H, W, w.shape[0])).copy()
    if taps == 1:
        return out + x @ w[:, 0, :].T
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        out += xp[1 + dy: 1 + dy + H, 1 + dx: 1 + dx + W, :] @ w[:, tap, :].T
    return out


def conv_backward(x, w, gout):
    """Gradients of conv: (d input, d w, d b) from d output."""
    H, W, _ = x.shape
    taps = w.shape[1]
    gb = gout.sum(axis=(0, 1))
    if taps == 1:
        gw = np.einsum("hwo,hwi->oi", gout, x)[:, None, :]
        return gout @ w[:, 0, :], gw, gb
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        xs = xp[1 + dy: 1 + dy + H, 1 + dx: 1 + dx + W, :]
        gw[:, tap, :] = np.einsum("hwo,hwi->oi", gout, xs)
        gxp[1 + dy: 1 + dy + H, 1 + dx: 1 + dx + W, :] += gout @ w[:, tap, :]
    return gxp[1:-1, 1:-1, :], gw, gb


def pool(x):
    """2 x 2 average pooling."""
    H, W, C = x.shape
    return x.reshape(H // 2, 2, W // 2, 2, C).mean(axis=(1, 3))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=0), 2, axis=1) * 0.25


def up(x):
    """Nearest 2x up-sampling."""
    return np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)


def up_backward(g):
    H, W, C = g.shape
    return g.reshape(H // 2, 2, W // 2, 2, C).sum(axis=(1, 3))


def relu(x):
    return np.maximum(x, 0.0)


# ---- network ----------------------------------------------------------
def forward(theta, x, bf16=False):
    """Returns the head output y (H, W, 16) and the stored activations."""
    q = to_bf16 if bf16 else (lambda a: a)
    L = [(q(w), b) for w, b in unpack(theta)]
    a = {"x": q(x), "L": L}
    a["e0"] = q(relu(conv(a["x"], *L[E[0]])))
    for lv in range(1, 5):
        a[f"p{lv - 1}"] = q(pool(a[f"e{lv - 1}"]))
        a[f"e{lv}"] = q(relu(conv(a[f"p{lv - 1}"], *L[E[lv]])))
    prev = a["e4"]
    for lv in (3, 2, 1, 0):
        a[f"c{lv}"] = np.concatenate([up(prev), a[f"e{lv}"]], axis=2)
        a[f"d{lv}"] = q(relu(conv(a[f"c{lv}"], *L[D[lv]])))
        prev = a[f"d{lv}"]
    y = conv(a["d0"], *L[HEAD])
    return y, a


def decode(y, d_lo, d_hi):
    """Head output -> inverse depths rho (H, W, K), raw directions m
    (H, W, K, 3), sigmoids."""
    rho_lo, rho_hi = 1.0 / d_hi, 1.0 / d_lo
    o = y.reshape(*y.shape[:2], K, 4)
    sig = 1.0 / (1.0 + np.exp(-o[..., 0]))
    return rho_lo + (rho_hi - rho_lo) * sig, o[..., 1:4], sig


def loss(y, target, mask, d_lo, d_hi, lam=LAMBDA_N):
    """Loss and its gradient with respect to y (min over the K proposals,
    averaged over all W x H pixels)."""
    H, W, _ = y.shape
    span = 1.0 / d_lo - 1.0 / d_hi
    rho, m, sig = decode(y, d_lo, d_hi)
    length = np.linalg.norm(m, axis=-1)
    n = m / length[..., None]
    rho_t = 1.0 / np.where(mask, target[..., 3], 1.0)
    nt = target[..., :3]
    dot = np.einsum("hwkc,hwc->hwk", n, nt)
    lk = np.abs(rho - rho_t[..., None]) / span + lam * (1.0 - np.abs(dot))
    best = np.argmin(lk, axis=2)                       # first minimum
    m_pix = mask.astype(bool)
    total = np.take_along_axis(lk, best[..., None], 2)[..., 0][m_pix].sum() / (W * H)
    g = np.zeros((H, W, K, 4))
    for yy, xx in zip(*np.nonzero(m_pix)):
        k = best[yy, xx]
        s = np.sign(rho[yy, xx, k] - rho_t[yy, xx])
        g[yy, xx, k, 0] = s * sig[yy, xx, k] * (1.0 - sig[yy, xx, k])
        d = dot[yy, xx, k]
        g[yy, xx, k, 1:] = -lam * np.sign(d) * (nt[yy, xx] - d * n[yy, xx, k]) / length[yy, xx, k]
    return total, g.reshape(H, W, 16) / (W * H)


def backward(theta, a, gy, bf16=False):
    """Gradient of the loss with respect to the flat parameters, from the
    activations of ``forward`` and d loss / d y."""
    q = to_bf16 if bf16 else (lambda v: v)
    L = a["L"]
    grads = [None] * len(LAYERS)
    gy = q(gy)
    gd, gw, gb = conv_backward(a["d0"], L[HEAD][0], gy)
    grads[HEAD] = (gw, gb)
    gd = q(gd)
    ge = {}
    for lv in (0, 1, 2, 3):
        gd = gd * (a[f"d{lv}"] > 0)
        gc, gw, gb = conv_backward(a[f"c{lv}"], L[D[lv]][0], gd)
        grads[D[lv]] = (gw, gb)
        gc = q(gc)
        up_ch = LAYERS[D[lv]][0] - LAYERS[E[lv]][1]
        ge[lv] = gc[..., up_ch:]
        gd = q(up_backward(gc[..., :up_ch]))         # gradient of d_{l+1} (or e_4)
    ge[4] = gd
    for lv in (4, 3, 2, 1, 0):
        g = ge[lv] * (a[f"e{lv}"] > 0)
        inp = a[f"p{lv - 1}"] if lv > 0 else a["x"]
        gi, gw, gb = conv_backward(inp, L[E[lv]][0], g)
        grads[E[lv]] = (gw, gb)
        if lv > 0:
            ge[lv - 1] = q(ge[lv - 1] + pool_backward(q(gi)))
    return pack(grads)


def loss_and_grad(theta, img, plane, cost, target, mask, d_lo, d_hi, bf16=False):
    x = make_input(img, plane, cost, d_lo, d_hi)
    y, a = forward(theta, x, bf16)
    total, gy = loss(y, target, mask, d_lo, d_hi)
    return total, backward(theta, a, gy, bf16), y


def propose(y, Kinv, d_lo, d_hi):
    """Head output -> (H, W, K, 4) planes (n, depth) with n . K^-1 x <= 0."""
    H, W, _ = y.shape
    rho, m, _ = decode(y, d_lo, d_hi)
    n = m / np.linalg.norm(m, axis=-1, keepdims=True)
    xs, ys = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ray = np.stack([xs, ys, np.ones_like(xs)], -1) @ np.asarray(Kinv, np.float64).T
    facing = np.einsum("hwkc,hwc->hwk", n, ray)
    n = np.where((facing > 0)[..., None], -n, n)
    return np.concatenate([n, (1.0 / rho)[..., None]], axis=-1)


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    return theta - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps), m, v
