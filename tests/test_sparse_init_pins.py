"""Pins of the sparse-feature depth initialisation oracle (Sec. III-B) to
closed forms (CPU only)."""
import numpy as np


class P:
    def __init__(self, **kw):
        self.win_radius, self.win_samples = 5.0, 6
        self.sigma_s, self.sigma_c = 5.0, 0.2
        self.d_lo, self.d_hi, self.seed = 2.0, 8.0, 11
        self.__dict__.update(kw)


def test_closest_feature_per_quadrant(oracle_lib):
    W, H = 40, 30                      # radius W / 10 = 4 px
    uv = [(22, 16), (18, 17), (17, 13), (22, 13)]     # quadrants 0..3 of pixel (20, 15), all within 4 px
    dep = [3.0, 4.0, 5.0, 6.0]
    rng = oracle_lib.sparse_range(W, H, uv, dep)
    assert tuple(rng[15, 20]) == (3.0, 6.0)
    # a closer feature in quadrant 0 replaces the one there
    rng = oracle_lib.sparse_range(W, H, uv + [(21, 15)], dep + [7.0])
    assert tuple(rng[15, 20]) == (4.0, 7.0)
    # features at the radius or beyond do not count; no feature: NaN
    rng = oracle_lib.sparse_range(W, H, [(24, 15), (20, 18.5)], [3.0, 5.0])
    assert tuple(rng[15, 20]) == (5.0, 5.0)
    assert np.isnan(rng[0, 0]).all()
    # depths outside the PatchMatch range are clamped into it
    rng = oracle_lib.sparse_range(W, H, [(21, 16), (19, 14)], [1.0, 9.5], d_lo=2.0, d_hi=8.0)
    assert tuple(rng[15, 20]) == (2.0, 8.0)
    # equal distances: the first listed feature wins
    rng = oracle_lib.sparse_range(W, H, [(21, 16), (21, 16)], [3.5, 6.5])
    assert tuple(rng[15, 20]) == (3.5, 3.5)


def test_fragile_choices_are_flagged(oracle_lib):
    """Pixel (20, 15), radius 4 px: a choice is flagged when a single-
    precision position or distance could decide it the other way — a
    feature 1e-6 px inside the radius, a feature 1e-6 px right of the pixel's
    column (quadrant 0 or 1), two features of one quadrant 1e-6 px apart in
    distance — and not flagged when every margin is above the band."""
    W, H = 40, 30
    firm = [(22.0, 16.0), (18.0, 17.0)]
    _, fr = oracle_lib.sparse_range(W, H, firm, [3.0, 4.0], band_px=1e-3, fragile=True)
    assert not fr[15, 20]
    for uv in ([(24.0 - 1e-6, 15.0)], [(20.0 + 1e-6, 17.0)], [(22.0, 16.0), (22.0 + 1e-6, 16.0)]):
        rng, fr = oracle_lib.sparse_range(W, H, uv, [3.0] * len(uv), band_px=1e-3, fragile=True)
        assert fr[15, 20] and not np.isnan(rng[15, 20]).any()
    # with no band nothing is flagged
    _, fr = oracle_lib.sparse_range(W, H, [(24.0 - 1e-6, 15.0)], [3.0], fragile=True)
    assert not fr.any()


def test_feature_filters_and_depth(oracle_lib):
    n = 3
    K = np.tile(np.array([[100.0, 0, 31.5], [0, 100.0, 23.5], [0, 0, 1]]), (n, 1, 1))
    R = np.tile(np.eye(3), (n, 1, 1))
    t = np.zeros((n, 3))
    t[:, 0] = [0.0, -0.2, -0.4]
    sc = oracle_lib.Scene(K, R, t, [np.zeros((48, 64), np.uint8)] * n)
    X = np.array([[0.1, 0.2, 4.0], [0.0, 0.0, 5.0], [0.3, -0.1, 6.0], [-0.2, 0.1, 3.0], [0.0, 0.1, 7.0]])
    vis = np.array([[1, 1, 1], [1, 1, 1], [1, 1, 0], [1, 0, 0], [0, 1, 1]], bool)
    reproj = np.array([0.5, 2.5, 1.0, 0.3, 0.2])
    obs = np.array([[34.0, 28.5], [31.5, 23.5], [36.5, 21.8], [24.8, 26.8], [0, 0]])
    uv, dep = oracle_lib.sparse_features(sc, 0, X, vis, reproj, obs, max_reproj=2.0)
    # mean views per point 11/5 = 2.2 -> at least floor(1.2) = 1 view; point 1
    # fails the re-projection error, point 4 is not visible in view 0; the
    # depth is the z of X in view 0 (R = I, t = 0 there)
    assert np.array_equal(dep, np.array([4.0, 6.0, 3.0]))
    assert np.array_equal(uv, np.array([[34.0, 28.5], [36.5, 21.8], [24.8, 26.8]]))
    # the depth in another view: z of X in view 1 (R = I, t = (-0.2, 0, 0))
    uv1, dep1 = oracle_lib.sparse_features(sc, 1, X, vis, reproj, obs, max_reproj=2.0)
    assert np.array_equal(dep1, np.array([4.0, 6.0, 7.0]))


def test_min_views_threshold(oracle_lib):
    n = 4
    K = np.tile(np.array([[100.0, 0, 31.5], [0, 100.0, 23.5], [0, 0, 1]]), (n, 1, 1))
    sc = oracle_lib.Scene(K, np.tile(np.eye(3), (n, 1, 1)), np.zeros((n, 3)), [np.zeros((48, 64), np.uint8)] * n)
    X = np.array([[0.0, 0.0, 4.0 + k] for k in range(4)])
    vis = np.array([[1, 1, 1, 1], [1, 1, 1, 1], [1, 1, 1, 1], [1, 0, 0, 0]], bool)
    # mean 13/4 = 3.25 -> floor(2.25) = 2: the point seen by one view goes
    uv, dep = oracle_lib.sparse_features(sc, 0, X, vis, np.zeros(4), np.zeros((4, 2)), max_reproj=2.0)
    assert np.array_equal(dep, np.array([4.0, 5.0, 6.0]))


def test_initialisation_draws_in_the_range(oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=40, H=30, n_src=2, seed=5)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    p = P()
    plain, _ = oracle_lib.init(osc, 0, [1, 2], p, with_cost=False)
    full = np.zeros((30, 40, 2), np.float32)
    full[..., 0], full[..., 1] = 2.0, 8.0
    same, _ = oracle_lib.init(osc, 0, [1, 2], p, with_cost=False, init_range=full)
    assert np.array_equal(same, plain)             # the range [d_lo, d_hi] is the plain draw
    point = np.full((30, 40, 2), 4.0, np.float32)
    pinned, _ = oracle_lib.init(osc, 0, [1, 2], p, with_cost=False, init_range=point)
    assert (pinned[..., 3] == 4.0).all() and np.array_equal(pinned[..., :3], plain[..., :3])
    rng = np.full((30, 40, 2), np.nan, np.float32)
    rng[10:20, 10:30] = (3.0, 5.0)
    mixed, _ = oracle_lib.init(osc, 0, [1, 2], p, with_cost=False, init_range=rng)
    u0 = (plain[..., 3] - 2.0) / 6.0               # the same Philox draw
    assert np.allclose(mixed[10:20, 10:30, 3], 3.0 + 2.0 * u0[10:20, 10:30], rtol=0, atol=1e-12)
    outside = np.isnan(rng[..., 0])
    assert np.array_equal(mixed[outside], plain[outside])
