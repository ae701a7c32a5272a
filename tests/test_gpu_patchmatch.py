"""GPU-vs-oracle parity of the PatchMatch path (through the C ABI).

Tolerances (stated by the build targets): per-pixel costs within 1e-4 of the
FP64 oracle; decisions (which candidate wins) identical outside the tie band
(gap between the two lowest competing costs < 2e-4) and outside fragile
discrete decisions (a window sample within 1e-3 px of a source border, a
weighted variance within 0.1 % of the flat limit).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

COST_TOL = 1e-4
TIE_BAND = 2e-4
MARGIN = 1e-3


@pytest.fixture(scope="module")
def small(mvs_lib, oracle_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=4, seed=7, baseline_frac=0.1)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, sigma_s=5.0, sigma_c=0.2, iters=3, seed=1234)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    yield sc, p, ctx, osc, [1, 2, 3, 4]
    ctx.close()


def _gpu_init(mvs, ctx, srcs, p):
    import copy
    q = copy.copy(p)
    q.iters, q.phase_begin, q.phase_end, q.init_mode = 0, 0, 0, mvs.MVS_INIT_RANDOM
    H, W = ctx.shapes[0]
    pl = np.zeros((H, W, 4), np.float32)
    co = np.zeros((H, W), np.float32)
    mvs.mvs_patchmatch(ctx.h, 0, srcs, q, pl, co)
    return pl, co


def test_plane_cost_parity_gt_and_random(small, mvs_lib, oracle_lib):
    sc, p, ctx, osc, srcs = small
    H, W = sc.gt_depth.shape
    gt = np.concatenate([sc.gt_normal, sc.gt_depth[..., None]], -1).astype(np.float32)
    rnd, _ = oracle_lib.init(osc, 0, srcs, p, with_cost=False)
    for planes in (gt, rnd.astype(np.float32)):
        cost = np.zeros((H, W), np.float32)
        vc = np.zeros((H, W, len(srcs)), np.float32)
        mvs_lib.mvs_plane_cost(ctx.h, 0, srcs, p, planes, cost, vc)
        oc, ovc, mg = oracle_lib.plane_cost(osc, 0, srcs, p, planes.astype(np.float64), with_views=True)
        firm = mg > MARGIN
        err = np.abs(cost - oc)
        assert err[firm].max() <= COST_TOL, f"max cost error {err[firm].max():.3g}"
        verr = np.abs(vc - ovc)
        assert verr[firm].max() <= COST_TOL, f"max per-view cost error {verr[firm].max():.3g}"
        assert (~firm).mean() < 0.01


def test_gt_planes_score_low_on_texture(small, mvs_lib):
    sc, p, ctx, osc, srcs = small
    H, W = sc.gt_depth.shape
    gt = np.concatenate([sc.gt_normal, sc.gt_depth[..., None]], -1).astype(np.float32)
    cost = np.zeros((H, W), np.float32)
    mvs_lib.mvs_plane_cost(ctx.h, 0, srcs, p, gt, cost)
    inner = np.zeros_like(sc.gt_textured)
    inner[8:-8, 8:-8] = True
    tex = sc.gt_textured & inner
    assert np.median(cost[tex]) < 0.05
    # pixels whose whole window lies on a texture-less quad: flat patch, C_max
    from scipy.ndimage import binary_erosion
    flat = binary_erosion(~sc.gt_textured, structure=np.ones((13, 13), bool))
    assert flat.sum() > 100 and (cost[flat] == 2.0).all()


def test_init_parity(small, mvs_lib, oracle_lib):
    sc, p, ctx, osc, srcs = small
    pl, co = _gpu_init(mvs_lib, ctx, srcs, p)
    opl, oco = oracle_lib.init(osc, 0, srcs, p)
    assert np.abs(pl[..., 3] - opl[..., 3]).max() <= 1e-6 * 8
    assert np.abs(pl[..., :3] - opl[..., :3]).max() <= 2e-6
    _, _, mg = oracle_lib.plane_cost(osc, 0, srcs, p, pl.astype(np.float64), with_views=True)
    firm = mg > MARGIN
    assert np.abs(co - oco)[firm].max() <= COST_TOL


def test_phase_lockstep(small, mvs_lib, oracle_lib):
    """Each half-iteration starts from the GPU's state on both sides."""
    import copy
    sc, p, ctx, osc, srcs = small
    pl, co = _gpu_init(mvs_lib, ctx, srcs, p)
    H, W = co.shape
    yy, xx = np.mgrid[0:H, 0:W]
    for ph in range(4):
        q = copy.copy(p)
        q.phase_begin, q.phase_end, q.init_mode = ph, ph + 1, mvs_lib.MVS_INIT_GIVEN
        g_pl, g_co = pl.copy(), co.copy()
        mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q, g_pl, g_co)
        o_pl, o_co, diag = oracle_lib.phase(osc, 0, srcs, p, ph, pl.astype(np.float64), co.astype(np.float64))
        other = ((xx + yy) & 1) != (ph & 1)
        # the other colour is untouched, bit for bit
        assert np.array_equal(g_pl[other], pl[other]) and np.array_equal(g_co[other], co[other])
        same = (np.abs(g_pl[..., 3] - o_pl[..., 3]) <= 1e-4 * o_pl[..., 3]) & \
               (np.abs(g_pl[..., :3] - o_pl[..., :3]).max(-1) <= 1e-3)
        tie = (diag["gap_prop"] < TIE_BAND) | (diag["gap_ref"] < TIE_BAND) | (diag["margin"] < MARGIN)
        active = ~other
        unexplained = active & ~same & ~tie
        assert unexplained.sum() == 0, f"phase {ph}: {unexplained.sum()} decisions differ outside the tie band"
        agree = active & same & (diag["margin"] >= MARGIN)
        assert np.abs(g_co - o_co)[agree].max() <= COST_TOL
        pl, co = g_pl, g_co


def test_resume_is_bit_identical(small, mvs_lib):
    import copy
    sc, p, ctx, osc, srcs = small
    H, W = sc.gt_depth.shape
    q = copy.copy(p)
    q.iters = 2
    a_pl = np.zeros((H, W, 4), np.float32)
    a_co = np.zeros((H, W), np.float32)
    mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q, a_pl, a_co)
    b_pl = np.zeros((H, W, 4), np.float32)
    b_co = np.zeros((H, W), np.float32)
    q1 = copy.copy(q)
    q1.phase_end = 1
    mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q1, b_pl, b_co)
    q2 = copy.copy(q)
    q2.phase_begin, q2.init_mode = 1, mvs_lib.MVS_INIT_GIVEN
    mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, q2, b_pl, b_co)
    assert np.array_equal(a_pl, b_pl) and np.array_equal(a_co, b_co)


def test_flat_pixels_keep_their_initial_plane(small, mvs_lib, oracle_lib):
    sc, p, ctx, osc, srcs = small
    H, W = sc.gt_depth.shape
    pl0, co0 = _gpu_init(mvs_lib, ctx, srcs, p)
    pl = np.zeros((H, W, 4), np.float32)
    co = np.zeros((H, W), np.float32)
    mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, p, pl, co)
    flat = co0 == 2.0
    # pixels whose reference patch is flat can never improve on C_max
    _, _, mg = oracle_lib.plane_cost(osc, 0, srcs, p, pl0.astype(np.float64), with_views=True)
    still = flat & (co == 2.0)
    assert np.array_equal(pl[still], pl0[still])


def test_free_running_depth(small, mvs_lib, oracle_lib):
    """Three free-running iterations: GPU vs oracle final depth."""
    sc, p, ctx, osc, srcs = small
    H, W = sc.gt_depth.shape
    pl = np.zeros((H, W, 4), np.float32)
    co = np.zeros((H, W), np.float32)
    mvs_lib.mvs_patchmatch(ctx.h, 0, srcs, p, pl, co)
    opl, oco = oracle_lib.patchmatch(osc, 0, srcs, p, p.iters)
    rel = np.abs(pl[..., 3] - opl[..., 3]) / opl[..., 3]
    frac = (rel <= 0.005).mean()
    print(f"free-running: depth within 0.5% on {frac:.5f} of pixels")
    assert frac >= 0.999        # measured 0.99943 on GB300
