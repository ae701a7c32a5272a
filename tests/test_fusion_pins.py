"""Pins of the depth-map fusion oracle (Sec. III-F) to closed forms and
invariants (CPU only).

The scene is a fronto-parallel plane z = d seen by cameras translated along
x by multiples of b, so that the projection of reference pixel (x, y) into
view k lands exactly on pixel (x - k s, y) with s = f b / d an integer: the
merges, the deletions and the counts then follow in closed form."""
import numpy as np

F, CX, CY = 100.0, 11.5, 3.5
W, H, D, B = 24, 8, 4.0, 0.2          # shift s = F * B / D = 5 px
S = int(round(F * B / D))


def _scene(oracle_lib, n_views):
    K = np.tile(np.array([[F, 0, CX], [0, F, CY], [0, 0, 1]], np.float64), (n_views, 1, 1))
    R = np.tile(np.eye(3), (n_views, 1, 1))
    # camera k at (k b, 0, 0): x_cam = X - C, so t = -C
    t = np.array([[-k * B, 0.0, 0.0] for k in range(n_views)])
    images = [np.zeros((H, W), np.uint8) for _ in range(n_views)]
    return oracle_lib.Scene(K, R, t, images)


def _plane(depth):
    pl = np.zeros((H, W, 4))
    pl[..., 2] = -1.0
    pl[..., 3] = depth
    return pl


def test_two_views_merge_in_closed_form(oracle_lib):
    sc = _scene(oracle_lib, 2)
    pts, sv, sp = oracle_lib.fuse(sc, [0, 1], {0: _plane(D), 1: _plane(D)})
    # view-0 pixel x merges with view-1 pixel x - s when x >= s
    assert len(pts) == 2 * H * W - H * (W - S)
    cnt0 = pts[sv == 0, 3].reshape(H, W)
    assert (cnt0[:, S:] == 2).all() and (cnt0[:, :S] == 1).all()
    # view 1 emits exactly its pixels that nobody claimed: x' >= W - s
    x1 = sp[sv == 1] % W
    assert sorted(set(x1.tolist())) == list(range(W - S, W))
    # every pixel ends in exactly one point
    assert pts[:, 3].sum() == 2 * H * W
    # merged points lie on the plane z = D, at the back-projection of the
    # emitting pixel (both members are the same 3D point)
    assert np.allclose(pts[:, 2], D, rtol=1e-6)
    xs = (sp[sv == 0] % W - CX) / F * D
    assert np.allclose(pts[sv == 0, 0], xs, atol=1e-5)


def test_relative_difference_threshold(oracle_lib):
    sc = _scene(oracle_lib, 2)
    # view 1's depth 2 % off: the pair differs by 0.02 d |ray| > 0.01 d
    pts, sv, _ = oracle_lib.fuse(sc, [0, 1], {0: _plane(D), 1: _plane(D * 1.02)})
    assert len(pts) == 2 * H * W and (pts[:, 3] == 1).all()
    # 0.5 % off: 0.005 d |ray| < 0.01 d, the same merges as exact maps
    pts, sv, _ = oracle_lib.fuse(sc, [0, 1], {0: _plane(D), 1: _plane(D * 1.005)})
    assert len(pts) == 2 * H * W - H * (W - S)
    # the average of d and 1.005 d along nearly the same ray
    assert np.allclose(pts[(sv == 0) & (pts[:, 3] == 2), 2], D * 1.0025, rtol=1e-5)


def test_order_and_deletion(oracle_lib):
    sc = _scene(oracle_lib, 3)
    planes = {v: _plane(D) for v in range(3)}
    pts, sv, sp = oracle_lib.fuse(sc, [0, 1, 2], planes)
    # view 0 pixel x takes view-1 pixel x - s and view-2 pixel x - 2s; view 1
    # keeps x' >= W - s, which merge with view-2 pixels x' - s; view 2 keeps
    # x'' >= W - s
    assert len(pts) == H * (W + 2 * S)
    cnt0 = pts[sv == 0, 3].reshape(H, W)
    assert (cnt0[:, :S] == 1).all() and (cnt0[:, S:2 * S] == 2).all() and (cnt0[:, 2 * S:] == 3).all()
    assert (pts[sv == 1, 3] == 2).all() and (pts[sv == 2, 3] == 1).all()
    assert pts[:, 3].sum() == 3 * H * W
    # the emitting view is the first in the processing order
    pts_r, sv_r, _ = oracle_lib.fuse(sc, [2, 1, 0], planes)
    assert len(pts_r) == len(pts) and (sv_r[: H * W] == 2).all()


def test_masks_and_missing_depth(oracle_lib):
    sc = _scene(oracle_lib, 2)
    p1 = _plane(D)
    p1[:, : W // 2, 3] = 0.0                       # no depth on the left half of view 1
    keep0 = np.ones((H, W), np.uint8)
    keep0[0] = 0                                   # first row of view 0 filtered out
    pts, sv, sp = oracle_lib.fuse(sc, [0, 1], {0: _plane(D), 1: p1}, keep={0: keep0})
    alive = (H - 1) * W + H * (W - W // 2)
    assert pts[:, 3].sum() == alive
    assert not np.isin(sp[sv == 0], np.arange(W)).any()
    # view-0 pixel x merges when its target x - s exists and has depth
    cnt0 = np.zeros((H, W))
    cnt0.ravel()[sp[sv == 0]] = pts[sv == 0, 3]
    assert (cnt0[1:, W // 2 + S:] == 2).all() and (cnt0[1:, : W // 2 + S] == 1).all()


def test_rigid_change_of_world_frame(oracle_lib):
    """Fusion does not depend on the world frame: with X' = Q X + T the
    cameras become R' = R Q^T, t' = t - R Q^T T and every point moves to
    Q X + T (pins the use of R versus R^T and of t)."""
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3))
    Q, _ = np.linalg.qr(A)
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    T = rng.normal(size=3) * 2.0
    n = 3
    K = np.tile(np.array([[F, 0, CX], [0, F, CY], [0, 0, 1]], np.float64), (n, 1, 1))
    R = np.tile(np.eye(3), (n, 1, 1))
    t = np.array([[-k * B, 0.0, 0.0] for k in range(n)])
    R2 = np.stack([R[k] @ Q.T for k in range(n)])
    t2 = np.stack([t[k] - R[k] @ Q.T @ T for k in range(n)])
    imgs = [np.zeros((H, W), np.uint8) for _ in range(n)]
    planes = {v: _plane(D) for v in range(n)}
    a = oracle_lib.fuse(oracle_lib.Scene(K, R, t, imgs), [0, 1, 2], planes)
    b = oracle_lib.fuse(oracle_lib.Scene(K, R2, t2, imgs), [0, 1, 2], planes)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]) and np.array_equal(a[0][:, 3], b[0][:, 3])
    moved = a[0][:, :3].astype(np.float64) @ Q.T + T
    assert np.allclose(b[0][:, :3], moved, atol=1e-4)


def test_fragile_rounding_follows_the_hint_and_firm_decisions_do_not(oracle_lib):
    """View 1 shifted by 5.5 - 1e-6 px: every projection of a view-0 pixel
    lands 1e-6 px past u + 1/2 = an integer, the boundary of the nearest-
    pixel rounding, where a single-precision computation may take either
    neighbour.  The oracle's own choice is floor(u + 1/2) (pixel x - 5);
    with a 1e-3 px band the decision is counted as fragile and a hint naming
    the other pixel (x - 6) is followed.  A hint that contradicts a firm decision (the 0.5 % depth
    offset of the other pins, no rounding boundary) changes nothing."""
    b2 = (5.5 - 1e-6) * D / F
    K = np.tile(np.array([[F, 0, CX], [0, F, CY], [0, 0, 1]], np.float64), (2, 1, 1))
    R = np.tile(np.eye(3), (2, 1, 1))
    t = np.array([[0.0, 0.0, 0.0], [-b2, 0.0, 0.0]])
    sc = oracle_lib.Scene(K, R, t, [np.zeros((H, W), np.uint8)] * 2)
    maps = {0: _plane(D), 1: _plane(D)}
    pts, sv, sp, own, st = oracle_lib.fuse(sc, [0, 1], maps, stats=True)
    assert st["fragile"] == 0
    own0 = own[: H * W].reshape(H, W)
    own1 = own[H * W:].reshape(H, W)
    # the oracle's own choice: view-0 pixel x takes view-1 pixel x - 5
    assert (own1[:, : W - 5] == own0[:, 5:]).all()
    _, _, _, own_b, st_b = oracle_lib.fuse(sc, [0, 1], maps, band_px=1e-3, stats=True)
    assert st_b["fragile"] == H * (W - 5) and st_b["resolved_by_hint"] == 0 and np.array_equal(own_b, own)
    # a hint in which view-0 pixel x took view-1 pixel x - 6 instead
    hint = np.full(2 * H * W, -1, np.int64)
    hint[: H * W] = np.arange(H * W)
    h1 = hint[H * W:].reshape(H, W)
    h1[:, : W - 6] = np.arange(H * W).reshape(H, W)[:, 6:]
    _, _, _, own_h, st_h = oracle_lib.fuse(sc, [0, 1], maps, band_px=1e-3, hint=hint, stats=True)
    own_h1 = own_h[H * W:].reshape(H, W)
    own_h0 = own_h[: H * W].reshape(H, W)
    assert (own_h1[:, : W - 6] == own_h0[:, 6:]).all()
    # ... and at x = 5, whose other candidate lies outside view 1, the hint's
    # "took nothing" is followed too
    assert st_h["resolved_by_hint"] == H * (W - 5)
    assert (own_h0[:, 5] != own_h1[:, 0]).all()
    # firm decisions ignore the hint
    sc1 = _scene(oracle_lib, 2)
    m2 = {0: _plane(D), 1: _plane(D * 1.005)}
    _, _, _, own_f, st_f = oracle_lib.fuse(sc1, [0, 1], m2, band_px=1e-3, band_rel=1e-3, stats=True)
    bogus = np.full(2 * H * W, -1, np.int64)
    _, _, _, own_g, st_g = oracle_lib.fuse(sc1, [0, 1], m2, band_px=1e-3, band_rel=1e-3, hint=bogus, stats=True)
    assert st_f["fragile"] == st_g["fragile"] == 0 and np.array_equal(own_f, own_g)
