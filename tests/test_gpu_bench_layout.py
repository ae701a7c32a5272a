"""Decision-level parity in the launch configurations the benchmarks time.

The reference is a 192 x 128 crop of the 3072 x 2048 high-resolution scene
(its principal point moved by the crop offset) and the sources are the ten
full-size views, so the phase kernel runs the layout of the measured
workload: 121-sample windows in 16-lane groups of 8 slots with ten sources
per pixel.  Each half-iteration starts from the GPU's state on both sides
(lockstep): the other colour is untouched, every decision agrees with the
FP64 oracle outside the tie band and the fragile-decision margin, costs and
per-view costs agree within 1e-4.  Two windows are checked: 21 x 21 at
dilation 2 (the benchmark's) and the paper's r_now / r_orig = 5 / 7
(s = 1.4, reference samples interpolated too).  The 16-slot layouts of the
undilated 15 x 15 and 21 x 21 windows (Table III's 7/7 and 10/10 rows) run
the same lockstep on the small scene, and 10/10 runs free as well.

Costs are compared for identical planes (the GPU's), with the tolerance
1e-4 on every view whose window image in the source is at most 256 px
across, and 1e-4 per 128 px of that extent beyond (grazing planes; the
count is printed and bounded)."""
import copy

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

COST_TOL = 1e-4
TIE_BAND = 2e-4
MARGIN = 1e-3
# Source positions are evaluated in float relative to the projected window
# centre, so their rounding grows with the extent of the window's image in
# the source (oracle.window_extent): about 2^-23 of it per sample, which the
# texture gradient turns into a cost error of a few 1e-7 per source pixel of
# extent.  Views up to EXTENT_PX across get COST_TOL; wider ones (grazing
# planes whose 21-pixel window spreads over hundreds of source pixels, 1-2 %
# of random initial planes) get COST_TOL per 128 px of extent (twice the
# largest error measured on GB300), and are counted.
EXTENT_PX = 256.0
WIDE_FRACTION = 0.03


def _view_tol(ext):
    return COST_TOL * np.maximum(1.0, ext / 128.0)
X0, Y0, CW, CH = 256, 1024, 192, 128      # crop of the 3072 x 2048 reference


@pytest.fixture(scope="module")
def crop_scene():
    from paper_2104_06165_gb300 import scenes
    sc = scenes.scene_highres(seed=0)
    K = sc.K.copy()
    K[0, 0, 2] -= X0
    K[0, 1, 2] -= Y0
    imgs = [np.ascontiguousarray(sc.images[0][Y0:Y0 + CH, X0:X0 + CW])] + list(sc.images[1:])
    tex = sc.gt_textured[Y0:Y0 + CH, X0:X0 + CW]
    return K, sc.R, sc.t, imgs, tex


def _params(mvs, r_orig, n, **kw):
    base = dict(win_radius=r_orig, win_samples=n, sigma_s=5.0, sigma_c=0.2, d_lo=2.0, d_hi=8.0, iters=1, seed=1)
    base.update(kw)
    return mvs.PMParams(**base)


def _lockstep(mvs, oracle, ctx, osc, srcs, p, n_phases):
    """Initial state, then n_phases half-iterations in lockstep; returns the
    per-phase counts for the report."""
    H, W = ctx.shapes[0]
    q = copy.copy(p)
    q.iters, q.phase_begin, q.phase_end, q.init_mode = 0, 0, 0, mvs.MVS_INIT_RANDOM
    pl = np.zeros((H, W, 4), np.float32)
    co = np.zeros((H, W), np.float32)
    mvs.mvs_patchmatch(ctx.h, 0, srcs, q, pl, co)
    opl, _ = oracle.init(osc, 0, srcs, p, with_cost=False)
    assert np.abs(pl[..., 3] - opl[..., 3]).max() <= 1e-6 * 8
    assert np.abs(pl[..., :3] - opl[..., :3]).max() <= 2e-6
    # costs of the same (float) planes on both sides: at 3072 px the float
    # rounding of a plane alone moves a far-off random plane's window by
    # ~1e-4 px in the source, so only identical planes give comparable costs
    _check_costs(mvs, oracle, ctx, osc, srcs, p, pl, co, np.ones(co.shape, bool), "init")
    yy, xx = np.mgrid[0:H, 0:W]
    report = []
    for ph in range(n_phases):
        q = copy.copy(p)
        q.phase_begin, q.phase_end, q.init_mode = ph, ph + 1, mvs.MVS_INIT_GIVEN
        g_pl, g_co = pl.copy(), co.copy()
        mvs.mvs_patchmatch(ctx.h, 0, srcs, q, g_pl, g_co)
        o_pl, o_co, diag = oracle.phase(osc, 0, srcs, p, ph, pl.astype(np.float64), co.astype(np.float64))
        other = ((xx + yy) & 1) != (ph & 1)
        assert np.array_equal(g_pl[other], pl[other]) and np.array_equal(g_co[other], co[other])
        active = ~other
        same = (np.abs(g_pl[..., 3] - o_pl[..., 3]) <= 1e-4 * o_pl[..., 3]) & \
               (np.abs(g_pl[..., :3] - o_pl[..., :3]).max(-1) <= 1e-3)
        tie = (diag["gap_prop"] < TIE_BAND) | (diag["gap_ref"] < TIE_BAND) | (diag["margin"] < MARGIN)
        unexplained = active & ~same & ~tie
        bad = np.argwhere(unexplained)[:5]
        detail = [(int(y), int(x), float(diag["gap_prop"][y, x]), float(diag["gap_ref"][y, x]),
                   float(diag["margin"][y, x]), float(g_co[y, x]), float(o_co[y, x])) for y, x in bad]
        assert unexplained.sum() == 0, f"phase {ph}: {unexplained.sum()} decisions differ outside the tie band: {detail}"
        # costs and per-view costs of the planes the GPU chose, on both sides
        # (the oracle's own choice differs from the GPU's plane by float
        # rounding, see above)
        _check_costs(mvs, oracle, ctx, osc, srcs, p, g_pl, g_co, active, f"phase {ph}")
        changed = active & ((g_pl != pl).any(-1))
        report.append((ph, int(active.sum()), int(changed.sum()), int((active & tie & ~same).sum()),
                       float((active & tie).mean())))
        pl, co = g_pl, g_co
    return report


def _check_costs(mvs, oracle, ctx, osc, srcs, p, pl, stored, sel, name):
    """Per-view and aggregated costs of the plane map pl on both sides, and
    the stored costs of the pixels in sel, within the extent-scaled tolerance
    wherever the oracle's decision margin is firm."""
    H, W = stored.shape
    vc = np.zeros((H, W, len(srcs)), np.float32)
    c2 = np.zeros((H, W), np.float32)
    mvs.mvs_plane_cost(ctx.h, 0, srcs, p, pl, c2, vc)
    f64 = pl.astype(np.float64)
    oc, ovc, mg = oracle.plane_cost(osc, 0, srcs, p, f64, with_views=True)
    ext = oracle.window_extent(osc, 0, srcs, p, f64)
    firm = mg > MARGIN
    tv = _view_tol(ext)
    tp = tv.max(-1)
    ev = np.abs(vc - ovc)
    ordinary = firm[..., None] & (ext <= EXTENT_PX)
    wide = firm[..., None] & (ext > EXTENT_PX)
    assert (ev[ordinary] <= COST_TOL).all()
    print(f"{name}: per-view cost error max {ev[ordinary].max():.2e} (p99.9 {np.quantile(ev[ordinary], 0.999):.2e}) "
          f"on {ordinary.sum()} views up to {EXTENT_PX:.0f} px; {wide.sum()} wider views, max error / tolerance "
          f"{(ev / tv)[wide].max() if wide.any() else 0.0:.2f}")
    assert (ev <= tv)[firm].all()
    assert (np.abs(c2 - oc) <= tp)[firm].all()
    assert (np.abs(stored - oc) <= tp)[firm & sel].all()
    assert wide.sum() <= WIDE_FRACTION * ordinary.sum()


@pytest.mark.parametrize("r_orig", [10.0, 7.0], ids=["21x21-dilation2", "paper-5-7"])
def test_phase_lockstep_at_the_benchmark_layout(crop_scene, mvs_lib, oracle_lib, r_orig):
    import torch
    K, R, t, imgs, tex = crop_scene
    srcs = list(range(1, 11))
    p = _params(mvs_lib, r_orig, 11)
    osc = oracle_lib.Scene(K, R, t, imgs)
    with mvs_lib.Context(K, R, t, imgs, stream=torch.cuda.current_stream()) as ctx:
        rep = _lockstep(mvs_lib, oracle_lib, ctx, osc, srcs, p, 2)
    for ph, act, chg, flips, tie_frac in rep:
        print(f"r_orig {r_orig}: phase {ph}: {act} active, {chg} changed, {flips} tie-band flips, "
              f"tie band {tie_frac:.4f}")
        assert chg > 0.3 * act          # the phase does real work on this crop


@pytest.fixture(scope="module")
def small_scene(mvs_lib, oracle_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=4, seed=7, baseline_frac=0.1)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    yield sc, ctx, osc
    ctx.close()


@pytest.mark.parametrize("r_orig, n", [(7.0, 15), (10.0, 21)], ids=["7-7-15x15", "10-10-21x21"])
def test_phase_lockstep_sixteen_slot_layouts(small_scene, mvs_lib, oracle_lib, r_orig, n):
    sc, ctx, osc = small_scene
    p = _params(mvs_lib, r_orig, n, seed=77)
    rep = _lockstep(mvs_lib, oracle_lib, ctx, osc, [1, 2, 3, 4], p, 2)
    for ph, act, chg, flips, tie_frac in rep:
        print(f"{n}x{n}: phase {ph}: {act} active, {chg} changed, {flips} tie-band flips, tie band {tie_frac:.4f}")


def test_free_running_sixteen_slot_layout(small_scene, mvs_lib, oracle_lib):
    """Three free-running iterations of the undilated 21 x 21 window: final
    depth within 0.5 % of the oracle's on at least 99.9 % of the pixels."""
    sc, ctx, osc = small_scene
    H, W = sc.gt_depth.shape
    p = _params(mvs_lib, 10.0, 21, iters=3, seed=5)
    pl = np.zeros((H, W, 4), np.float32)
    co = np.zeros((H, W), np.float32)
    mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2, 3, 4], p, pl, co)
    opl, oco = oracle_lib.patchmatch(osc, 0, [1, 2, 3, 4], p, 3)
    frac = (np.abs(pl[..., 3] - opl[..., 3]) <= 0.005 * opl[..., 3]).mean()
    print(f"21x21 free-running: depth within 0.5% on {frac:.5f} of pixels")
    assert frac >= 0.999


@pytest.mark.parametrize("which", ["crop", "small"])
def test_candidate_memo_is_exact(crop_scene, small_scene, mvs_lib, which):
    """Within one call the phase kernel does not score again a propagated
    plane that a pixel scored (or found equal to a scored one) at its
    previous visit.  Running the same phases as separate one-phase calls
    (the memo starts empty in every call) gives the same plane and cost maps
    bit for bit, with more ZNCC evaluations."""
    import torch
    if which == "crop":
        K, R, t, imgs, _ = crop_scene
        ctx = mvs_lib.Context(K, R, t, imgs, stream=torch.cuda.current_stream())
        srcs, p = list(range(1, 11)), _params(mvs_lib, 10.0, 11, iters=4, seed=3)
    else:
        sc, ctx, _ = small_scene
        srcs, p = [1, 2, 3, 4], _params(mvs_lib, 5.0, 6, iters=4, seed=3)
    try:
        H, W = ctx.shapes[0]
        mvs_lib.mvs_profile(ctx.h, 1)
        a_pl = np.zeros((H, W, 4), np.float32)
        a_co = np.zeros((H, W), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, p, a_pl, a_co)
        ev_one = mvs_lib.mvs_profile_read(ctx.h)[3]
        mvs_lib.mvs_profile(ctx.h, 1)
        b_pl = np.zeros((H, W, 4), np.float32)
        b_co = np.zeros((H, W), np.float32)
        q = copy.copy(p)
        q.iters, q.phase_begin, q.phase_end = 0, 0, 0
        mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q, b_pl, b_co)
        for ph in range(2 * p.iters):
            q = copy.copy(p)
            q.phase_begin, q.phase_end, q.init_mode = ph, ph + 1, mvs_lib.MVS_INIT_GIVEN
            mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q, b_pl, b_co)
        ev_sep = mvs_lib.mvs_profile_read(ctx.h)[3]
        mvs_lib.mvs_profile(ctx.h, 0)
    finally:
        if which == "crop":
            ctx.close()
    assert np.array_equal(a_pl, b_pl) and np.array_equal(a_co, b_co)
    print(f"{which}: {ev_one} ZNCC evaluations in one call, {ev_sep} in one-phase calls "
          f"({1 - ev_one / ev_sep:.1%} skipped)")
    assert ev_one < ev_sep
