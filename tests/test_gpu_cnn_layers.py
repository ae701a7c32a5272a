"""Layer-by-layer (lockstep) parity of the proposal network's kernels.

After one forward and backward pass the library's stored tensors are read
back (mvs_cnn_read).  Each convolution is then recomputed by the FP64 oracle
from the library's own stored input (bf16) and the bf16 weights, so that the
comparison covers exactly one kernel launch and no earlier rounding:

* bf16 outputs (activations, data gradients): the library stores the fp32
  sum rounded to bf16.  Where the exact value lies farther from a bf16
  rounding midpoint than the fp32 accumulation error can reach, that must be
  bf16(exact) bit for bit; elsewhere the neighbouring bf16 value is also a
  correct answer.  The accumulation error is bounded by
  (ceil(K / 8) + 4) 2^-23 sum |terms| for a K-term dot product (one
  rounding per tensor-core k-step, with room for the steps' internal
  alignment); a value off bf16(exact) must lie within one bf16 step of the
  exact value and have its exact value within that bound of the midpoint.
  At least 99.9 % of the elements must be bit-exact.
* fp32 outputs (head output, weight and bias gradients): within
  (n + 2) 2^-23 sum |terms|, twice the bound of recursive summation of n
  terms (n: the longest chain of dependent additions the kernel performs;
  the factor two allows truncating tensor-core additions).
Pooling, up-sampling, concatenation and the ReLU masks are exact
operations on bf16 values and are compared bit for bit.

Cases: 64 x 48 and 768 x 32 (the widest training size; its rows span many
pixel tiles and its smallest level is 48 x 2)."""
import math

import numpy as np
import pytest

from oracle import cnn_oracle as cn

pytestmark = pytest.mark.gpu

D_LO, D_HI = 2.0, 8.0
ENC = [0, 1, 2, 3, 4]
DEC = {3: 5, 2: 6, 1: 7, 0: 8}


def _state(rng, W, H):
    img = rng.integers(20, 236, (H, W)).astype(np.uint8)
    n = rng.normal(0, 1, (H, W, 3))
    n[..., 2] = -np.abs(n[..., 2]) - 1.0
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    plane = np.concatenate([n, rng.uniform(D_LO, D_HI, (H, W, 1))], -1).astype(np.float32)
    cost = rng.uniform(0, 2, (H, W)).astype(np.float32)
    return img, plane, cost


def _bf16_step(v):
    """Spacing of bfloat16 numbers at |v| (8 significant bits)."""
    _, e = np.frexp(np.abs(v))
    return np.ldexp(1.0, e - 8)


def _check_bf16(name, got, v, abssum, K, stats, relu=False, mask=None):
    """got: the library's stored bf16 values of bf16(act(v')) (times mask),
    v' its fp32 sum; v: the exact sum.  Rounding is monotonic, so with
    |v' - v| <= b every correct result lies in [r(v - b), r(v + b)], r the
    bf16 rounding after the activation; and bf16(act(v)) is expected on all
    but a small fraction."""
    b = (math.ceil(K / 8) + 4) * 2.0 ** -23 * abssum
    act = cn.relu if relu else (lambda t: t)
    msk = 1.0 if mask is None else mask
    lo = cn.to_bf16(act(v - b)) * msk
    hi = cn.to_bf16(act(v + b)) * msk
    inside = (got >= np.minimum(lo, hi)) & (got <= np.maximum(lo, hi))
    assert inside.all(), (f"{name}: {(~inside).sum()} values outside every correct rounding, e.g. "
                          f"{got[~inside][:3]} for exact {v[~inside][:3]}")
    frac = (got == cn.to_bf16(act(v)) * msk).mean()
    stats.append((name, got.size, frac))
    assert frac >= 0.999, f"{name}: only {frac:.5f} bit-exact"


def _check_f32(name, got, exact, abssum, n_chain):
    # 2^-23 per addition: tensor-core sums may truncate instead of rounding
    bound = (n_chain + 2) * 2.0 ** -23 * abssum + 1e-30
    err = np.abs(got.astype(np.float64) - exact)
    assert (err <= bound).all(), f"{name}: max error / bound {(err / bound).max():.3g}"


def _conv_abs(x, w, b):
    return cn.conv(np.abs(x), np.abs(w), np.abs(b))


@pytest.mark.parametrize("W, H", [(64, 48), (768, 32)])
def test_every_layer_in_lockstep(mvs_lib, W, H):
    import torch
    m = mvs_lib
    rng = np.random.default_rng(W + H)
    img, plane, cost = _state(rng, W, H)
    _, target, _ = _state(rng, W, H)
    mask = (rng.uniform(size=(H, W)) < 0.7).astype(np.uint8)
    net = m.mvs_cnn_create(W, H, D_LO, D_HI, 31, torch.cuda.current_stream())
    stats = []
    try:
        theta = m.mvs_cnn_get_params(net).astype(np.float64)
        off = 0
        for ci, co, t in cn.LAYERS:      # biases with a spread, as in a trained network
            off += co * t * ci
            theta[off: off + co] = rng.normal(0, 0.05, co)
            off += co
        m.mvs_cnn_set_params(net, theta.astype(np.float32))
        theta = m.mvs_cnn_get_params(net).astype(np.float64)
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (img, plane, cost, target, mask)]
        m.mvs_cnn_backward(net, *dev)
        torch.cuda.synchronize()
        rd = lambda t, lv=0: m.mvs_cnn_read(net, t, lv, W, H).astype(np.float64)
        L = [(cn.to_bf16(w), b) for w, b in cn.unpack(theta)]
        grads = cn.unpack(m.mvs_cnn_get_grads(net).astype(np.float64))

        # ---- forward ----
        x = rd(m.MVS_CNN_T_INPUT)
        xin = cn.make_input(img, plane.astype(np.float64), cost.astype(np.float64), D_LO, D_HI)
        # the input is a few fp32 operations per value: bit-exact unless within
        # their rounding of a bf16 midpoint
        _check_bf16("input", x, xin, 8.0 * np.maximum(np.abs(xin), 1.0), 1, stats)
        e = {}
        for lv in range(5):
            inp = x if lv == 0 else rd(m.MVS_CNN_T_POOL, lv - 1)
            if lv > 0:
                assert np.array_equal(inp, cn.to_bf16(cn.pool(e[lv - 1]))), f"pool {lv - 1}"
            w, b = L[ENC[lv]]
            e[lv] = rd(m.MVS_CNN_T_ENC, lv)
            _check_bf16(f"e{lv}", e[lv], cn.conv(inp, w, b), _conv_abs(inp, w, b), 9 * w.shape[2], stats, relu=True)
        prev = e[4]
        d = {}
        cat = {}
        for lv in (3, 2, 1, 0):
            cat[lv] = rd(m.MVS_CNN_T_CAT, lv)
            assert np.array_equal(cat[lv], np.concatenate([cn.up(prev), e[lv]], axis=2)), f"cat {lv}"
            w, b = L[DEC[lv]]
            d[lv] = rd(m.MVS_CNN_T_DEC, lv)
            _check_bf16(f"d{lv}", d[lv], cn.conv(cat[lv], w, b), _conv_abs(cat[lv], w, b), 9 * w.shape[2], stats,
                        relu=True)
            prev = d[lv]
        w, b = L[9]
        y = rd(m.MVS_CNN_T_HEAD)
        _check_f32("head", y, cn.conv(d[0], w, b), _conv_abs(d[0], w, b), 32 + 1)

        # ---- backward (data gradients) ----
        gy = rd(m.MVS_CNN_T_GRAD_HEAD)
        _, gy_exact = cn.loss(y, target.astype(np.float64), mask, D_LO, D_HI)
        # the library's loss gradient is fp32 (its own kernel): within one bf16
        # step wherever the fp32 and fp64 minima over the K proposals agree
        near = np.abs(gy - gy_exact) <= _bf16_step(gy_exact) + 1e-12
        assert near.mean() >= 0.9999, f"head gradient: {near.mean():.6f} within one bf16 step"
        K = 16
        gd = rd(m.MVS_CNN_T_GRAD_DEC, 0)
        gx = gy @ w[:, 0, :]
        _check_bf16("gd0", gd, gx, np.abs(gy) @ np.abs(w[:, 0, :]), K, stats, mask=(d[0] > 0))
        gdec = {0: gd}
        for lv in (0, 1, 2, 3):
            w, _ = L[DEC[lv]]
            gc = rd(m.MVS_CNN_T_GRAD_CAT, lv)
            gxe, _, _ = cn.conv_backward(cat[lv], w, gdec[lv])
            gxa, _, _ = cn.conv_backward(cat[lv], np.abs(w), np.abs(gdec[lv]))
            _check_bf16(f"gc{lv}", gc, gxe, gxa, 9 * w.shape[0], stats)
            up_ch = cn.LAYERS[DEC[lv]][0] - cn.LAYERS[ENC[lv]][1]
            nxt = cn.to_bf16(cn.up_backward(gc[..., :up_ch]))
            if lv < 3:
                gdec[lv + 1] = rd(m.MVS_CNN_T_GRAD_DEC, lv + 1)
                assert np.array_equal(gdec[lv + 1], nxt * (d[lv + 1] > 0)), f"gd{lv + 1}"
            else:
                genc4 = nxt
        ge = {lv: rd(m.MVS_CNN_T_GRAD_ENC, lv) for lv in range(5)}
        assert np.array_equal(ge[4], genc4 * (e[4] > 0)), "ge4"
        for lv in (4, 3, 2, 1):
            w, _ = L[ENC[lv]]
            gp = rd(m.MVS_CNN_T_GRAD_POOL, lv - 1)
            inp = rd(m.MVS_CNN_T_POOL, lv - 1)
            gxe, _, _ = cn.conv_backward(inp, w, ge[lv])
            gxa, _, _ = cn.conv_backward(inp, np.abs(w), np.abs(ge[lv]))
            _check_bf16(f"gp{lv - 1}", gp, gxe, gxa, 9 * w.shape[0], stats)
            gc = rd(m.MVS_CNN_T_GRAD_CAT, lv - 1)
            up_ch = cn.LAYERS[DEC[lv - 1]][0] - cn.LAYERS[ENC[lv - 1]][1]
            skip = gc[..., up_ch:]
            expect = cn.to_bf16(skip + cn.pool_backward(gp)) * (e[lv - 1] > 0)
            assert np.array_equal(ge[lv - 1], expect), f"ge{lv - 1}"

        # ---- weight and bias gradients ----
        gouts = {9: gy}
        ins = {9: d[0]}
        for lv in range(4):
            gouts[DEC[lv]], ins[DEC[lv]] = gdec[lv], cat[lv]
        for lv in range(5):
            gouts[ENC[lv]] = ge[lv]
            ins[ENC[lv]] = x if lv == 0 else rd(m.MVS_CNN_T_POOL, lv - 1)
        rows = 4
        for li in range(10):
            w = L[li][0]
            _, gw, gb = cn.conv_backward(ins[li], w, gouts[li])
            _, gwa, gba = cn.conv_backward(np.abs(ins[li]), w, np.abs(gouts[li]))
            hh, ww_ = ins[li].shape[:2]
            chain = rows * ww_ + (hh + rows - 1) // rows
            _check_f32(f"grad w {li}", grads[li][0], gw, gwa, chain)
            _check_f32(f"grad b {li}", grads[li][1], gb, gba, chain)
    finally:
        m.mvs_cnn_destroy(net)
    for name, n, frac in stats:
        print(f"{W}x{H} {name}: {n} values, {frac:.6f} bit-exact")


def test_bounded_wait_reports_timeout_and_recovers(mvs_lib):
    """A convolution whose wait targets a barrier that nothing completes gives
    up after its bound and reports MVS_ETIMEOUT once; the network then runs
    normally (the same forward pass gives the same head output as before)."""
    import torch
    m = mvs_lib
    W, H = 64, 48
    rng = np.random.default_rng(3)
    img, plane, cost = _state(rng, W, H)
    net = m.mvs_cnn_create(W, H, D_LO, D_HI, 5, torch.cuda.current_stream())
    try:
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (img, plane, cost)]
        out0 = torch.zeros((H, W, 16), dtype=torch.float32, device="cuda")
        m.mvs_cnn_forward(net, *dev, out0)
        torch.cuda.synchronize()
        assert m.mvs_cnn_test_timeout(net) == m.MVS_ETIMEOUT
        assert m.mvs_cnn_test_timeout(net) == m.MVS_ETIMEOUT        # each check reports its own
        out1 = torch.zeros_like(out0)
        m.mvs_cnn_forward(net, *dev, out1)
        m.mvs_cnn_get_params(net)                                    # synchronises: no pending timeout
        assert torch.equal(out0, out1)
    finally:
        m.mvs_cnn_destroy(net)
