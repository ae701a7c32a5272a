"""Pins of the neighbouring-image selection oracle (Sec. III-A, Eqs. 1-3) to
closed forms of simple camera layouts (CPU only)."""
import math

import numpy as np

Z = 5.0


def _grid_points(n=10):
    g = np.linspace(-0.8, 0.8, n)
    xx, yy = np.meshgrid(g, g)
    return np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, Z)], 1)


def test_tau_closed_form_for_parallel_cameras(oracle_lib):
    """Reference at the origin, sources shifted by b along x, all looking
    along +z, points on the plane z = Z: the disturbance of Eq. 1 moves every
    projection into source j by f b eps / ((1 + eps) Z) along x (Eq. 2)."""
    f, eps = 400.0, 0.002
    bs = [0.0, 0.2, 0.5, 1.0]
    n = len(bs)
    K = np.tile(np.array([[f, 0, 399.5], [0, f, 299.5], [0, 0, 1]]), (n, 1, 1))
    R = np.tile(np.eye(3), (n, 1, 1))
    t = np.array([[-b, 0.0, 0.0] for b in bs])
    sc = oracle_lib.Scene(K, R, t, [np.zeros((600, 800), np.uint8)] * n)
    X = _grid_points()
    vis = np.ones((len(X), n), bool)
    nbr, tau, na, zeta = oracle_lib.select_neighbors(sc, X, vis, eps=eps, t_tau=0.0, k=3)
    for j in range(1, n):
        assert math.isclose(tau[0, j], f * bs[j] * eps / ((1 + eps) * Z), rel_tol=1e-9)
        assert na[0, j] == len(X)


def _ring(alphas_deg, f=1000.0):
    """Reference on the optical axis through (0, 0, Z); sources at angle
    alpha from it on a circle of radius Z around (0, 0, Z), all looking at
    that point: principal-axis angle alpha, baseline 2 Z sin(alpha / 2)."""
    from paper_2104_06165_gb300 import scenes
    Ks, Rs, ts = [], [], []
    for a in [0.0] + list(alphas_deg):
        r = math.radians(a)
        C = np.array([0.0, 0.0, Z]) + Z * np.array([math.sin(r), 0.0, -math.cos(r)])
        R, t = scenes.look_at(C, [0.0, 0.0, Z])
        Ks.append(np.array([[f, 0, 499.5], [0, f, 499.5], [0, 0, 1]]))
        Rs.append(R)
        ts.append(t)
    return np.stack(Ks), np.stack(Rs), np.stack(ts)


def test_ranking_by_shared_points_and_tau_filter(oracle_lib):
    """With b > 0.1 and theta > 0.05 for every source, Eq. 3 reduces to
    0.005 / N_A: the eight sources sharing the most points win, most first.
    A source almost at the reference (0.5 degrees) shares every point and
    would rank first, but its tau is below t_tau and removes it."""
    alphas = [10, 15, 20, 25, 30, 35, 40, 45, 50, 0.5]
    shared = [30, 80, 50, 90, 10, 70, 60, 20, 40, 100]
    K, R, t = _ring(alphas)
    n = len(alphas) + 1
    sc = oracle_lib.Scene(K, R, t, [np.zeros((1000, 1000), np.uint8)] * n)
    X = _grid_points()
    vis = np.zeros((len(X), n), bool)
    vis[:, 0] = True
    for j, m in enumerate(shared, start=1):
        vis[:m, j] = True
    nbr, tau, na, zeta = oracle_lib.select_neighbors(sc, X, vis, k=8)
    expect = [1 + j for j in sorted(range(9), key=lambda j: -shared[j])][:8]
    assert nbr[0].tolist() == expect
    assert tau[0, 10] < 0.1 and np.isinf(zeta[0, 10]) and na[0, 10] == 100
    assert (tau[0, 1:10] > 0.1).all()
    for j in range(1, 10):
        assert math.isclose(zeta[0, j], 0.1 * 0.05 / shared[j - 1], rel_tol=1e-12)


def test_small_angle_is_not_truncated(oracle_lib):
    """A source at 2 degrees (theta = 0.0349 rad < 0.05, baseline 0.17 > 0.1)
    keeps its own angle in Eq. 3: zeta = 0.1 theta / N_A, which puts it ahead
    of a source sharing more points.  The focal length is that of a
    3072-pixel-wide image, where Eq. 2 moves its projections by 0.2 px,
    above Sec. IV's t_tau = 0.1."""
    alphas = [2.0, 20.0, 30.0]
    shared = [80, 100, 60]
    K, R, t = _ring(alphas, f=2880.0)
    n = len(alphas) + 1
    sc = oracle_lib.Scene(K, R, t, [np.zeros((1000, 1000), np.uint8)] * n)
    X = _grid_points()
    vis = np.zeros((len(X), n), bool)
    vis[:, 0] = True
    for j, m in enumerate(shared, start=1):
        vis[:m, j] = True
    nbr, tau, na, zeta = oracle_lib.select_neighbors(sc, X, vis, k=8)
    assert tau[0, 1] > 0.1
    th = math.radians(2.0)
    assert math.isclose(zeta[0, 1], 0.1 * th / 80, rel_tol=1e-9)
    # 0.1 * 0.0349 / 80 < 0.005 / 100 < 0.005 / 60; truncating theta to 0.05
    # as well would give 0.005 / 80 and the order 2, 1, 3
    assert nbr[0, :3].tolist() == [1, 2, 3] and nbr[0, 3] == -1
    # the symmetric pair shares the same points
    assert na[1, 0] == na[0, 1] == 80


def test_defaults_are_the_papers():
    """The oracle's and the binding's defaults for Eq. 1's eps and Eq. 2's
    t_tau are the values Sec. IV gives (tests/golden/paper_constants.json),
    and so are the C header's named constants."""
    import inspect
    import json
    import os
    import re

    import oracle
    from paper_2104_06165_gb300 import mvs
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "tests", "golden", "paper_constants.json")) as fh:
        pc = json.load(fh)
    for fn in (oracle.select_neighbors, mvs.mvs_select_neighbors):
        sig = inspect.signature(fn)
        assert sig.parameters["eps"].default == pc["epsilon"]
        assert sig.parameters["t_tau"].default == pc["t_tau"]
    assert inspect.signature(oracle.select_neighbors).parameters["k"].default == 8
    with open(os.path.join(root, "include", "mvs.h")) as fh:
        hdr = fh.read()
    assert float(re.search(r"#define MVS_NBR_EPS ([0-9.]+)", hdr).group(1)) == pc["epsilon"]
    assert float(re.search(r"#define MVS_NBR_T_TAU ([0-9.]+)", hdr).group(1)) == pc["t_tau"]
