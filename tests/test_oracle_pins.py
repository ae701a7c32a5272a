"""Pins of the FP64 oracle to things other than itself: library routines,
closed forms, brute force and invariants the paper fixes (CPU only)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


class P:
    """Parameter record (the oracle reads these attribute names)."""

    def __init__(self, **kw):
        self.win_radius, self.win_samples = 5.0, 6
        self.sigma_s, self.sigma_c = 5.0, 0.2
        self.d_lo, self.d_hi, self.seed = 2.0, 8.0, 1
        self.__dict__.update(kw)


# --------------------------------------------------------------------------
# Philox4x64-10 against numpy's implementation (library routine)
# --------------------------------------------------------------------------
def test_philox_matches_numpy(oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(50):
        ctr = [int(x) for x in rng.integers(0, 2 ** 63, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 63, 2)]
        bg = np.random.Philox(counter=ctr, key=key)
        ref = [int(x) for x in bg.random_raw(4)]
        # numpy advances the counter by one before producing the block
        c1 = list(ctr)
        c1[0] = (c1[0] + 1) & (2 ** 64 - 1)
        assert oracle_lib.philox4x64(c1, key) == ref


def test_init_draws_are_uniform(oracle_lib):
    """Sec. III-B draws: depth uniform in [d_lo, d_hi] (chi-square), normals
    facing the camera with unit length."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=64, H=48, n_src=1, seed=0)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    pl, _ = oracle_lib.init(osc, 0, [1], P(seed=99), with_cost=False)
    d = pl[..., 3].ravel()
    assert d.min() >= 2.0 and d.max() < 8.0
    hist, _ = np.histogram(d, bins=16, range=(2, 8))
    exp = d.size / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 40.0   # 15 dof, p ~ 5e-4
    n = pl[..., :3]
    assert np.allclose(np.linalg.norm(n, axis=-1), 1.0, atol=1e-12)
    Kinv = np.linalg.inv(sc.K[0])
    yy, xx = np.mgrid[0:48, 0:64]
    rays = np.stack([xx, yy, np.ones_like(xx)], -1) @ Kinv.T
    assert (np.sum(n * rays, -1) <= 0).all()


# --------------------------------------------------------------------------
# bilinear interpolation and the dilated window (Sec. III-C)
# --------------------------------------------------------------------------
def test_bilinear_exact_on_affine_images(oracle_lib):
    H, W = 7, 9
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    img = 0.3 + 0.01 * xx - 0.02 * yy
    rng = np.random.default_rng(1)
    for _ in range(200):
        u, v = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        assert abs(oracle_lib.bilinear(img, u, v) - (0.3 + 0.01 * u - 0.02 * v)) < 1e-14
    img2 = rng.uniform(0, 1, (H, W))
    for y in range(H):
        for x in range(W):
            assert oracle_lib.bilinear(img2, x, y) == img2[y, x]


def test_window_offsets(oracle_lib):
    assert np.allclose(oracle_lib.window_offsets(P(win_radius=5.0, win_samples=6)), [-5, -3, -1, 1, 3, 5])
    assert np.allclose(oracle_lib.window_offsets(P(win_radius=10.0, win_samples=11)), np.arange(-10, 11, 2))
    # the paper's default r_now / r_orig = 5 / 7: scale s = 1.4, non-integer samples
    assert np.allclose(oracle_lib.window_offsets(P(win_radius=7.0, win_samples=11)), 1.4 * np.arange(-5, 6))


# --------------------------------------------------------------------------
# plane-induced homography (Sec. III-C)
# --------------------------------------------------------------------------
def _two_view(R, t, W=40, H=30, f=50.0):
    import oracle
    K = np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1.0]])
    img = np.zeros((H, W))
    return oracle.Scene(np.stack([K, K]), np.stack([np.eye(3), R]), np.stack([np.zeros(3), t]), [img, img]), K


def test_homography_fronto_parallel_closed_form(oracle_lib):
    b, d, f = 0.3, 4.0, 50.0
    osc, K = _two_view(np.eye(3), np.array([-b, 0.0, 0.0]), f=f)
    Hm = oracle_lib.homography(osc, 0, 1, 10, 12, np.array([0.0, 0.0, -1.0]), d)
    for (u, v) in [(0, 0), (10, 12), (33.5, 7.25), (39, 29)]:
        q = Hm @ np.array([u, v, 1.0])
        assert abs(q[0] / q[2] - (u - f * b / d)) < 1e-12 and abs(q[1] / q[2] - v) < 1e-12


def test_homography_equals_point_transfer(oracle_lib):
    """H maps a pixel to the projection of the back-projected point on the
    plane, for random poses and planes."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.normal(size=3) * 0.2
        th = np.linalg.norm(a)
        k = a / th
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
        t = rng.normal(size=3) * 0.3
        osc, K = _two_view(R, t)
        x, y = int(rng.integers(0, 40)), int(rng.integers(0, 30))
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        r = np.linalg.inv(K) @ np.array([x, y, 1.0])
        if n @ r > 0:
            n = -n
        d = rng.uniform(2, 8)
        Hm = oracle_lib.homography(osc, 0, 1, x, y, n, d)
        rho = n @ (d * r)
        for _ in range(5):
            e = np.array([rng.uniform(0, 39), rng.uniform(0, 29), 1.0])
            re = np.linalg.inv(K) @ e
            X = re * rho / (n @ re)          # ray-plane intersection
            Xs = R @ X + t
            p = K @ Xs
            q = Hm @ e
            assert np.allclose(q[:2] / q[2], p[:2] / p[2], atol=1e-9)


# --------------------------------------------------------------------------
# ZNCC (Eq. 4) and aggregation (Eq. 5)
# --------------------------------------------------------------------------
def test_weighted_zncc_matches_numpy(oracle_lib):
    rng = np.random.default_rng(5)
    for _ in range(50):
        m = int(rng.integers(4, 60))
        w = rng.uniform(0.01, 1, m)
        a, b = rng.uniform(0, 1, m), rng.uniform(0, 1, m)
        c = np.cov(a, b, aweights=w)
        assert abs(oracle_lib.wzncc(w, a, b) - c[0, 1] / math.sqrt(c[0, 0] * c[1, 1])) < 1e-12
        assert abs(oracle_lib.wzncc(w, a, 2.5 * a + 0.3) - 1.0) < 1e-12      # affine, alpha > 0: Z = 1
        assert abs(oracle_lib.wzncc(w, a, -0.5 * a + 0.9) + 1.0) < 1e-12     # alpha < 0: Z = -1
        assert abs(oracle_lib.wzncc(np.ones(m), a, b) - np.corrcoef(a, b)[0, 1]) < 1e-12   # Eq. 4 unweighted


def test_aggregation_is_weighted_harmonic_mean(oracle_lib):
    from scipy.stats import hmean
    rng = np.random.default_rng(6)
    for _ in range(50):
        nv = int(rng.integers(1, 10))
        c = rng.uniform(0.01, 1.99, nv)
        ok = rng.integers(0, 2, nv)
        agg = oracle_lib.aggregate(c, ok)
        sel = c[ok == 1]
        if sel.size == 0:
            assert agg == 2.0
        else:
            assert abs(agg - hmean(sel)) < 1e-12
    assert oracle_lib.aggregate([2.0, 2.0], [1, 1]) == 2.0      # C_max views are left out
    assert abs(oracle_lib.aggregate([0.0, 0.5], [1, 1]) - 2 / (1e6 + 2)) < 1e-15


def test_identical_views_cost_zero(oracle_lib):
    """A source identical to the reference (same camera, same image): every
    plane maps each sample to itself, Z = 1, C = the 1e-6 floor."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=48, H=36, n_src=1, seed=2, baseline=0.0)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    rng = np.random.default_rng(0)
    n = np.concatenate([rng.uniform(-0.5, 0.5, (36, 48, 2)), -np.ones((36, 48, 1))], -1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    pl = np.concatenate([n, rng.uniform(2, 8, (36, 48, 1))], -1)
    c = oracle_lib.plane_cost(osc, 0, [1], P(), pl)
    assert (c[8:-8, 8:-8] <= 1e-6).all()


def test_flat_and_out_of_border_give_cmax(oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=48, H=36, n_src=1, seed=2, textured=False)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    pl = np.zeros((36, 48, 4))
    pl[..., 2] = -1
    pl[..., 3] = 4.0
    assert (oracle_lib.plane_cost(osc, 0, [1], P(), pl) == 2.0).all()
    sc2 = scenes.make_plane_scene(W=48, H=36, n_src=1, seed=2, baseline=8.0)   # disparity > width: leaves the image
    osc2 = oracle_lib.Scene(sc2.K, sc2.R, sc2.t, sc2.images)
    assert (oracle_lib.plane_cost(osc2, 0, [1], P(), pl) == 2.0).all()


def test_ground_truth_plane_is_a_sharp_minimum(oracle_lib):
    """Unquantised render of one slanted textured plane: the true plane
    scores near zero and beats +-0.5 % depth and 3 degree tilts."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=64, H=48, n_src=2, seed=4, depth=4.0, normal=(0.2, -0.1, -1.0),
                                 quantise=False, lam_px=(6.0, 24.0))
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    gt = np.concatenate([sc.gt_normal, sc.gt_depth[..., None]], -1)
    c0 = oracle_lib.plane_cost(osc, 0, [1, 2], P(), gt)[10:-10, 10:-10]
    assert np.median(c0) < 2e-3
    for s in (0.995, 1.005):
        g2 = gt.copy()
        g2[..., 3] *= s
        c = oracle_lib.plane_cost(osc, 0, [1, 2], P(), g2)[10:-10, 10:-10]
        assert (c > c0).mean() > 0.97


# --------------------------------------------------------------------------
# propagation pattern and phases (Sec. III, III-C)
# --------------------------------------------------------------------------
def test_group_members_are_other_colour(oracle_lib):
    sizes = []
    for g in range(8):
        m = oracle_lib.group_members(g)
        sizes.append(len(m))
        assert ((np.abs(m).sum(1) % 2) == 1).all()       # odd |dx|+|dy|: the other colour
        assert (np.abs(m).max() <= 25)
    assert sizes == [6, 6, 6, 6, 11, 11, 11, 11]
    up = {tuple(r) for r in oracle_lib.group_members(0)}
    assert {(-dy, dx) for dx, dy in up} == {tuple(r) for r in oracle_lib.group_members(3)}


@pytest.fixture(scope="module")
def tiny(oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=40, H=30, n_src=2, seed=11, baseline_frac=0.1, n_textured=1, n_flat=1)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    return sc, osc


def test_phase_touches_one_colour_and_never_raises_cost(oracle_lib, tiny):
    sc, osc = tiny
    p = P(seed=3)
    pl, co = oracle_lib.init(osc, 0, [1, 2], p)
    yy, xx = np.mgrid[0:30, 0:40]
    for ph in range(4):
        pl2, co2, diag = oracle_lib.phase(osc, 0, [1, 2], p, ph, pl, co)
        other = ((xx + yy) & 1) != (ph & 1)
        assert np.array_equal(pl2[other], pl[other]) and np.array_equal(co2[other], co[other])
        assert (co2 <= co).all()
        # the stored cost is the cost of the stored plane
        assert np.allclose(oracle_lib.plane_cost(osc, 0, [1, 2], p, pl2)[~other], co2[~other], atol=1e-12)
        pl, co = pl2, co2


def test_patchmatch_equals_init_plus_phases(oracle_lib, tiny):
    sc, osc = tiny
    p = P(seed=8)
    a_pl, a_co = oracle_lib.patchmatch(osc, 0, [1, 2], p, 2)
    pl, co = oracle_lib.init(osc, 0, [1, 2], p)
    for ph in range(4):
        pl, co, _ = oracle_lib.phase(osc, 0, [1, 2], p, ph, pl, co)
    assert np.array_equal(a_pl, pl) and np.array_equal(a_co, co)


def test_proposals_outside_the_depth_range_change_nothing(oracle_lib, tiny):
    sc, osc = tiny
    p = P(seed=4)
    pl, co = oracle_lib.init(osc, 0, [1, 2], p)
    props = np.zeros((30, 40, 3, 4))
    props[..., 2] = -1.0
    props[..., 0, 3] = 0.0          # unused slot
    props[..., 1, 3] = 1.9          # below d_lo
    props[..., 2, 3] = 8.5          # above d_hi
    for ph in range(2):
        a_pl, a_co, a_d = oracle_lib.phase(osc, 0, [1, 2], p, ph, pl, co)
        b_pl, b_co, b_d = oracle_lib.phase(osc, 0, [1, 2], p, ph, pl, co, proposals=props)
        assert np.array_equal(a_pl, b_pl) and np.array_equal(a_co, b_co)
        assert np.array_equal(a_d["win_prop"], b_d["win_prop"])
        pl, co = a_pl, a_co


def test_ground_truth_proposals_are_taken(oracle_lib):
    """On a single textured plane the true plane offered as a proposal wins
    wherever it is cheaper than what propagation found; the phase's cost is
    then at most the true plane's cost (refinement only lowers it)."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=32, H=24, n_src=2, seed=12, depth=4.0, normal=(0.2, -0.1, -1.0), f=60.0,
                                 baseline=0.25)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    p = P(seed=6, win_radius=3.0, win_samples=4)
    pl, co = oracle_lib.init(osc, 0, [1, 2], p)
    gt = np.concatenate([sc.gt_normal, sc.gt_depth[..., None]], -1)
    gt_cost = oracle_lib.plane_cost(osc, 0, [1, 2], p, gt)
    rng = np.random.default_rng(0)
    props = np.zeros((24, 32, 2, 4))
    props[..., 0, :] = gt
    props[..., 1, :3] = [0.0, 0.0, -1.0]
    props[..., 1, 3] = rng.uniform(2.0, 8.0, (24, 32))
    yy, xx = np.mgrid[0:24, 0:32]
    mine = ((xx + yy) & 1) == 0
    pl2, co2, d = oracle_lib.phase(osc, 0, [1, 2], p, 0, pl, co, proposals=props)
    assert (co2[mine] <= gt_cost[mine] + 1e-12).all()
    took_gt = d["win_prop"] == 8
    assert took_gt[mine].mean() > 0.5
    kept = took_gt & mine & (d["win_ref"] < 0)        # no refinement candidate replaced it
    assert kept.any() and np.allclose(pl2[kept], gt[kept], atol=1e-12)


def test_patchmatch_reaches_exhaustive_search_minimum(oracle_lib):
    """Tiny scene of one slanted plane: after 6 iterations PatchMatch's cost
    is within 1e-3 of (or below) the best of an exhaustive search over 48
    depths x 81 normals on the textured interior."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=20, H=16, n_src=2, seed=9, depth=4.0, normal=(0.15, 0.1, -1.0), f=40.0,
                                 baseline=0.25)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    p = P(seed=5, win_radius=3.0, win_samples=4)
    _, co = oracle_lib.patchmatch(osc, 0, [1, 2], p, 6)
    best = np.full((16, 20), np.inf)
    Kinv = np.linalg.inv(sc.K[0])
    for th in np.linspace(-0.3, 0.3, 9):
        for ph in np.linspace(-0.3, 0.3, 9):
            n = np.array([math.sin(th), math.sin(ph), -1.0])
            n /= np.linalg.norm(n)
            for d in np.linspace(2.0, 8.0, 48):
                pl = np.zeros((16, 20, 4))
                pl[..., :3] = n
                pl[..., 3] = d
                best = np.minimum(best, oracle_lib.plane_cost(osc, 0, [1, 2], p, pl))
    inner = (slice(4, -4), slice(4, -4))
    assert (co[inner] <= best[inner] + 1e-3).mean() > 0.9


# --------------------------------------------------------------------------
# geometric consistency (Sec. III-D)
# --------------------------------------------------------------------------
def test_geo_filter_keeps_consistent_and_drops_shifted(oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=48, H=36, n_src=3, seed=3, depth=4.0, normal=(0.1, 0.0, -1.0), baseline=0.15)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    planes = {}
    for v in range(4):
        out = scenes.render(sc.quads, sc.K[v], sc.R[v], sc.t[v], 48, 36, want_gt=True, threads=1)
        planes[v] = np.concatenate([out["normal"], out["depth"][..., None]], -1)
    keep, cnt = oracle_lib.geo_filter(osc, 0, [1, 2, 3], planes)
    inner = (slice(6, -6), slice(6, -6))
    assert keep[inner].all() and (cnt[inner] == 3).all()
    shifted = {v: (pl.copy() if v == 0 else pl + np.array([0, 0, 0, 0.03])) for v, pl in planes.items()}
    keep2, _ = oracle_lib.geo_filter(osc, 0, [1, 2, 3], shifted)
    assert not keep2.any()
    one = dict(planes)
    one[2] = planes[2] + np.array([0, 0, 0, 0.03])
    one[3] = planes[3] + np.array([0, 0, 0, 0.03])
    keep3, cnt3 = oracle_lib.geo_filter(osc, 0, [1, 2, 3], one)
    assert not keep3.any() and (cnt3[inner] == 1).all()     # "more than one" view needed
    # the decision margin follows the depth test: sources 5e-6 beyond the
    # 0.02 tolerance (band 1e-5) make every interior pixel fragile, sources
    # 0.01 beyond it almost none
    for dz, fragile in ((0.020005, 1.0), (0.03, 0.0)):
        sh = {v: (pl.copy() if v == 0 else pl + np.array([0, 0, 0, dz])) for v, pl in planes.items()}
        _, _, mg = oracle_lib.geo_filter(osc, 0, [1, 2, 3], sh, with_margin=True)
        assert abs((mg[inner] < 1.0).mean() - fragile) < 0.05


# --------------------------------------------------------------------------
# PHI (Sec. III-E)
# --------------------------------------------------------------------------
def _nearest6_fit(depth, known, x, y, k, n_fit=6):
    """Brute force: sort the reconstructed pixels of the line by (distance,
    side) and fit with numpy.polyfit."""
    H, W = depth.shape
    dx, dy = [(1, 0), (0, 1), (1, 1), (1, -1)][k]
    pts = []
    for t in range(-max(W, H), max(W, H) + 1):
        if t == 0:
            continue
        qx, qy = x + t * dx, y + t * dy
        if 0 <= qx < W and 0 <= qy < H and known[qy, qx]:
            pts.append((abs(t), 0 if t < 0 else 1, t, depth[qy, qx]))
    pts.sort()
    pts = pts[:n_fit]
    if len(pts) < 2:
        return None
    t = np.array([p[2] for p in pts], float)
    v = np.array([p[3] for p in pts], float)
    return np.polyfit(t, v, 1)[1]


def test_line_fit_matches_polyfit_on_nearest_six(oracle_lib):
    rng = np.random.default_rng(12)
    H, W = 14, 17
    depth = rng.uniform(2, 8, (H, W))
    known = (rng.uniform(size=(H, W)) < 0.4).astype(np.uint8)
    for _ in range(150):
        x, y, k = int(rng.integers(0, W)), int(rng.integers(0, H)), int(rng.integers(0, 4))
        if known[y, x]:
            continue
        ref = _nearest6_fit(depth, known, x, y, k)
        got = oracle_lib.line_fit_at(depth, known, x, y, k, d_lo=-1e9, d_hi=1e9)
        if ref is None:
            assert got is None
        else:
            assert abs(got - ref) < 1e-9


def test_line_fit_fills_linear_depth_exactly(oracle_lib):
    H, W = 20, 30
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    depth = 3.0 + 0.05 * xx + 0.02 * yy           # linear along every line direction
    known = np.ones((H, W), np.uint8)
    known[5:15, 8:22] = 0
    hyp, valid = oracle_lib.phi_hypotheses(depth * known, known, d_lo=0, d_hi=100)
    hole = known == 0
    for k in range(4):
        v = valid[..., k].astype(bool) & hole
        assert np.allclose(hyp[..., k][v], depth[v], atol=1e-10)
    assert valid[hole].all()


def test_potentials_ranges(oracle_lib):
    k1, k2, k3 = 4.0, 0.5, 2.0
    for c in np.linspace(0, 2, 21):
        u = oracle_lib.phi_unary(c, k1, k2)
        assert k2 - 1e-15 <= u <= 2 / k1 + k2 + 1e-15
    rng = np.random.default_rng(2)
    for _ in range(200):
        a, b = rng.uniform(0.5, 10, 2)
        e = oracle_lib.phi_pair(a, b, k3)
        assert (k3 - 1) ** 2 - 1e-12 <= e <= k3 ** 2 + 1e-12
        assert e == oracle_lib.phi_pair(b, a, k3)
    assert oracle_lib.phi_pair(3.0, 3.0, k3) == 4.0
    assert oracle_lib.phi_pair(2.0, 5.0, k3) == 1.0


def _random_mrf(rng, gh, gw, L, scale_un=1.0):
    nlab = rng.integers(1, L + 1, (gh, gw)).astype(np.int32)
    lab = rng.uniform(2, 8, (gh, gw, 4))
    un = rng.uniform(0, 0.7, (gh, gw, 4)) * scale_un
    return nlab, lab, un


def _brute(nlab, lab, un, k3=2.0):
    gh, gw = nlab.shape
    best, arg = np.inf, None
    for ls in itertools.product(*[range(int(n)) for n in nlab.ravel()]):
        lb = np.array(ls, np.int32).reshape(gh, gw)
        e = 0.0
        for y in range(gh):
            for x in range(gw):
                e += un[y, x, lb[y, x]]
                if x + 1 < gw:
                    e -= math.log((k3 - min(1, abs(lab[y, x, lb[y, x]] - lab[y, x + 1, lb[y, x + 1]]) /
                                            min(lab[y, x, lb[y, x]], lab[y, x + 1, lb[y, x + 1]]))) ** 2)
                if y + 1 < gh:
                    e -= math.log((k3 - min(1, abs(lab[y, x, lb[y, x]] - lab[y + 1, x, lb[y + 1, x]]) /
                                            min(lab[y, x, lb[y, x]], lab[y + 1, x, lb[y + 1, x]]))) ** 2)
        if e < best - 1e-12:
            best, arg = e, lb
    return best, arg


def test_mrf_energy_matches_brute_force_formula(oracle_lib):
    rng = np.random.default_rng(4)
    for _ in range(20):
        nlab, lab, un = _random_mrf(rng, 2, 3, 3)
        lb = np.array([[rng.integers(0, n) for n in row] for row in nlab], np.int32)
        e_or = oracle_lib.mrf_energy(nlab, lab, un, lb)
        # recompute with the brute-force helper restricted to this labelling
        one = np.ones_like(nlab)
        lab2 = np.take_along_axis(lab, lb[..., None], 2)
        un2 = np.take_along_axis(un, lb[..., None], 2)
        e_b, _ = _brute(one, np.repeat(lab2, 4, 2), np.repeat(un2, 4, 2))
        assert abs(e_or - e_b) < 1e-10


def test_trw_is_exact_on_chains(oracle_lib):
    """On a chain TRW-S (node weight 1) is exact min-sum dynamic programming:
    the decoded labelling is the enumerated MAP."""
    rng = np.random.default_rng(7)
    for _ in range(30):
        n = int(rng.integers(2, 8))
        nlab, lab, un = _random_mrf(rng, 1, n, 4)
        label, _ = oracle_lib.trw(nlab, lab, un, iters=1)
        e_star, arg = _brute(nlab, lab, un)
        assert abs(oracle_lib.mrf_energy(nlab, lab, un, label) - e_star) < 1e-9
    for _ in range(10):                        # vertical chains too
        n = int(rng.integers(2, 7))
        nlab, lab, un = _random_mrf(rng, n, 1, 3)
        label, _ = oracle_lib.trw(nlab, lab, un, iters=1)
        e_star, _ = _brute(nlab, lab, un)
        assert abs(oracle_lib.mrf_energy(nlab, lab, un, label) - e_star) < 1e-9


def test_trw_on_small_grids_is_near_the_map(oracle_lib):
    rng = np.random.default_rng(8)
    exact = 0
    for _ in range(20):
        nlab, lab, un = _random_mrf(rng, 3, 3, 3)
        label, _ = oracle_lib.trw(nlab, lab, un, iters=10)
        e_star, _ = _brute(nlab, lab, un)
        e = oracle_lib.mrf_energy(nlab, lab, un, label)
        assert e >= e_star - 1e-9
        exact += abs(e - e_star) < 1e-9
    assert exact >= 16


def test_eq10_normal_of_a_planar_depth_map(oracle_lib):
    from paper_2104_06165_gb300 import scenes
    n_true = np.array([0.3, -0.2, -1.0])
    n_true /= np.linalg.norm(n_true)
    sc = scenes.make_plane_scene(W=30, H=20, n_src=1, seed=1, depth=5.0, normal=n_true)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    for (x, y) in [(5, 5), (15, 10), (28, 18)]:
        n = oracle_lib.eq10_normal(osc, 0, sc.gt_depth, x, y)
        assert np.allclose(n, n_true, atol=1e-9)
    assert oracle_lib.eq10_normal(osc, 0, sc.gt_depth, 0, 5) is None


def test_plane_infer_fills_a_hole_in_a_fronto_parallel_plane(oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=40, H=30, n_src=2, seed=6, depth=5.0, normal=(0, 0, -1.0), baseline=0.2)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    plane = np.concatenate([sc.gt_normal, sc.gt_depth[..., None]], -1)
    known = np.ones((30, 40), np.uint8)
    known[8:20, 10:25] = 0
    plane[known == 0] = 0
    out, aux = oracle_lib.plane_infer(osc, 0, [1, 2], P(), known, plane)
    filled = aux["filled"].astype(bool)
    assert filled[9:19, 11:24].all()
    assert np.allclose(out[..., 3][filled], 5.0, atol=1e-9)
    assert np.allclose(out[..., :3][filled], [0, 0, -1], atol=1e-9)


def test_paper_constants_fixture():
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as f:
        g = json.load(f)
    from paper_2104_06165_gb300.mvs import PMParams, PhiParams, FilterParams
    p, q, f_ = PMParams(), PhiParams(), FilterParams()
    r_now = (p.win_samples - 1) / 2
    assert (r_now, p.win_radius) == (g["r_now"], g["r_orig"])
    assert (q.kappa1, q.kappa2, q.kappa3) == (g["kappa1"], g["kappa2"], g["kappa3"])
    assert p.iters == g["iterations"] and q.trw_iters == g["trw_iterations"] and q.n_fit == g["n_fit"]
    assert (f_.depth_tol, f_.max_angle_deg, f_.max_reproj_px) == (g["filter_depth"], g["filter_angle_deg"],
                                                                  g["filter_reproj_px"])


def test_cost_at_equals_the_cost_map(oracle_lib, tiny):
    sc, osc = tiny
    p = P(seed=2)
    pl, _ = oracle_lib.init(osc, 0, [1, 2], p)
    full = oracle_lib.plane_cost(osc, 0, [1, 2], p, pl)
    xs = np.array([0, 5, 39, 20, 11])
    ys = np.array([0, 7, 29, 15, 3])
    c, _ = oracle_lib.cost_at(osc, 0, [1, 2], p, xs, ys, pl[ys, xs])
    assert np.array_equal(c, full[ys, xs])


# --------------------------------------------------------------------------
# PHI-MVS/M (Sec. IV, Table I): the MRF removed, each hole takes its valid
# hypothesis of minimal matching cost
# --------------------------------------------------------------------------
def test_min_cost_selection_is_masked_argmin_and_recovers_the_plane(oracle_lib):
    from phi_cases import slanted_hole_case
    rng = np.random.default_rng(21)
    sc, n_true, known, hyp, valid, hcost, plane, best = slanted_hole_case(rng)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    out, filled = oracle_lib.phi_select_min_cost(osc, 0, known, hyp, valid, hcost, plane)
    # library routine: numpy's argmin (first minimum) over the masked costs
    k = np.argmin(np.where(valid == 1, hcost, np.inf), axis=-1)
    assert np.array_equal(k[known == 0], best[known == 0])
    hole = known == 0
    f = filled.astype(bool)
    assert f[hole].all() and not f[~hole].any()
    # the exact planar depth is chosen everywhere, so Eq. 10 gives the plane normal
    assert np.allclose(out[..., 3][f], sc.gt_depth[f], rtol=0, atol=1e-12)
    assert np.allclose(out[..., :3][f], n_true, atol=1e-9)
    assert np.array_equal(out[~hole], plane[~hole])


def test_min_cost_selection_empty_holes(oracle_lib):
    from phi_cases import slanted_hole_case
    rng = np.random.default_rng(5)
    sc, n_true, known, hyp, valid, hcost, plane, best = slanted_hole_case(rng)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    valid[10, 12] = 0                      # no hypothesis: stays empty, and so do
    out, filled = oracle_lib.phi_select_min_cost(osc, 0, known, hyp, valid, hcost, plane)
    assert (out[10, 12] == 0).all() and not filled[10, 12]
    # its four neighbours lack one Eq. 10 neighbour and stay empty too
    for (y, x) in [(9, 12), (11, 12), (10, 11), (10, 13)]:
        assert (out[y, x] == 0).all() and not filled[y, x]


def test_plane_infer_min_cost_fills_a_fronto_parallel_hole(oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=40, H=30, n_src=2, seed=6, depth=5.0, normal=(0, 0, -1.0), baseline=0.2)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    plane = np.concatenate([sc.gt_normal, sc.gt_depth[..., None]], -1)
    known = np.ones((30, 40), np.uint8)
    known[8:20, 10:25] = 0
    plane[known == 0] = 0
    out, aux = oracle_lib.plane_infer(osc, 0, [1, 2], P(), known, plane, min_cost=True)
    filled = aux["filled"].astype(bool)
    assert filled[9:19, 11:24].all()
    assert np.allclose(out[..., 3][filled], 5.0, atol=1e-9)
    assert np.allclose(out[..., :3][filled], [0, 0, -1], atol=1e-9)
    assert (aux["label"] == -3).all()
    # the same intermediates, selected by minimal cost
    sel, _ = oracle_lib.phi_select_min_cost(osc, 0, known, aux["hyp"], aux["valid"], aux["hcost"], plane)
    assert np.array_equal(sel, out)


def test_min_cost_and_mrf_selections_agree_with_one_hypothesis_per_hole(oracle_lib):
    """With exactly one valid hypothesis in every hole (so no MRF node lacks
    a label) both selections must take it: the MRF pipeline and PHI-MVS/M
    give the same map, whatever the costs."""
    from phi_cases import slanted_hole_case
    rng = np.random.default_rng(9)
    sc, n_true, known, hyp, valid, hcost, plane, best = slanted_hole_case(rng)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    H, W = known.shape
    pick = rng.integers(0, 4, (H, W))           # a random, generally perturbed, hypothesis
    one = np.zeros_like(valid)
    yy, xx = np.mgrid[0:H, 0:W]
    one[yy, xx, pick] = 1
    depth = plane[..., 3]
    label, _ = oracle_lib.phi_mrf(known, depth, hyp, one, hcost)
    assert (label[known[::2, ::2] == 0] >= 0).all()
    a, fa = oracle_lib.phi_select(osc, 0, known, hyp, one, label, plane)
    b, fb = oracle_lib.phi_select_min_cost(osc, 0, known, hyp, one, hcost, plane)
    assert np.array_equal(fa, fb) and fa[known == 0].mean() > 0.5
    assert np.array_equal(a, b)
    chosen = hyp[yy, xx, pick]
    assert np.array_equal(b[..., 3][fb == 1], chosen[fb == 1])


def test_window_extent_closed_forms(oracle_lib):
    """Window extent diagnostic: a fronto-parallel plane seen by an x-shifted
    copy of the camera maps the window by a pure translation, so the extent
    is the largest sample offset (5 px for 6 x 6 samples at dilation 2); a
    source camera with twice the focal length doubles it; an unusable plane
    (facing away) gives 0."""
    b, d, f = 0.3, 4.0, 50.0
    osc, K = _two_view(np.eye(3), np.array([-b, 0.0, 0.0]), f=f)
    p = P(win_radius=5.0, win_samples=6)
    plane = np.zeros((30, 40, 4))
    plane[..., 2], plane[..., 3] = -1.0, d
    ext = oracle_lib.window_extent(osc, 0, [1], p, plane)[..., 0]
    assert np.allclose(ext[10:20, 10:30], 5.0, atol=1e-12)
    assert (ext[0, 0] >= 0) and ext.max() <= 5.0 + 1e-12     # border windows lose samples
    K2 = K.copy()
    K2[0, 0] = K2[1, 1] = 2 * f
    osc2 = oracle_lib.Scene(np.stack([K, K2]), np.stack([np.eye(3)] * 2), np.stack([np.zeros(3), [-b, 0.0, 0.0]]),
                            [np.zeros((30, 40))] * 2)
    ext2 = oracle_lib.window_extent(osc2, 0, [1], p, plane)[..., 0]
    assert np.allclose(ext2[10:20, 10:30], 10.0, atol=1e-12)
    away = plane.copy()
    away[..., 2] = 1.0
    assert (oracle_lib.window_extent(osc, 0, [1], p, away) == 0).all()
