"""PHI-MVS/M (Sec. IV, Table I: plane hypothesis inference with the MRF
removed, each hole taking its hypothesis of minimal matching cost) on the GPU
against the oracle, and the Table I comparison of PatchMatch alone, PHI-MVS/M
and PHI-MVS on a synthetic scene with texture-less regions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx(mvs_lib, sc):
    import torch
    return mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())


def test_min_cost_select_equals_oracle_on_planted_hypotheses(mvs_lib, oracle_lib):
    """Slanted plane, exact hypothesis at the lowest cost (ties planted at a
    higher index): identical choices, the exact depth, the plane normal."""
    import torch
    from phi_cases import slanted_hole_case
    rng = np.random.default_rng(21)
    sc, n_true, known, hyp, valid, hcost, plane, best = slanted_hole_case(rng)
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    ctx = _ctx(mvs_lib, sc)
    try:
        gpl = f32(plane)
        mvs_lib.mvs_phi_select_min_cost(ctx.h, 0, known, f32(hyp), valid, f32(hcost), gpl)
        # device buffers give the same map
        dpl = torch.from_numpy(f32(plane)).cuda()
        mvs_lib.mvs_phi_select_min_cost(ctx.h, 0, torch.from_numpy(known).cuda(), torch.from_numpy(f32(hyp)).cuda(),
                                        torch.from_numpy(valid).cuda(), torch.from_numpy(f32(hcost)).cuda(), dpl)
        assert np.array_equal(dpl.cpu().numpy(), gpl)
    finally:
        ctx.close()
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    # the oracle decides on the same single-precision hypotheses and costs
    opl, ofilled = oracle_lib.phi_select_min_cost(osc, 0, known, f32(hyp).astype(np.float64), valid,
                                                  f32(hcost).astype(np.float64), f32(plane).astype(np.float64))
    f = ofilled.astype(bool)
    assert f.sum() == (known == 0).sum()
    assert np.array_equal((gpl[..., 3] > 0) & (known == 0), f)
    assert np.array_equal(gpl[..., 3][f], opl[..., 3][f].astype(np.float32))      # same choice, bit for bit
    assert np.array_equal(gpl[..., 3][f], f32(sc.gt_depth)[f])
    assert np.abs(gpl[..., :3][f] - n_true).max() < 1e-4
    assert np.array_equal(gpl[known == 1], f32(plane)[known == 1])


def test_min_cost_select_equals_oracle_on_line_fit_hypotheses(mvs_lib, oracle_lib):
    """Oracle hypotheses and costs of a rendered scene with holes, cast to
    single precision and given to both selections."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=128, H=96, n_src=3, seed=21, baseline_frac=0.1)
    out = scenes.render(sc.quads, sc.K[0], sc.R[0], sc.t[0], 128, 96, want_gt=True, threads=1)
    gt = np.concatenate([out["normal"], out["depth"][..., None]], -1)
    rng = np.random.default_rng(8)
    known = (gt[..., 3] > 0).astype(np.uint8)
    known[20:60, 30:90] = 0
    known[rng.uniform(size=known.shape) < 0.15] = 0
    plane = gt * known[..., None]
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    ohyp, ovalid = oracle_lib.phi_hypotheses(plane[..., 3], known, d_lo=2.0, d_hi=8.0)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6)
    ocost = oracle_lib.phi_cost(osc, 0, [1, 2, 3], p, ohyp, ovalid)
    h32, c32 = np.ascontiguousarray(ohyp, np.float32), np.ascontiguousarray(ocost, np.float32)
    opl, ofilled = oracle_lib.phi_select_min_cost(osc, 0, known, h32.astype(np.float64), ovalid,
                                                  c32.astype(np.float64), plane)
    ctx = _ctx(mvs_lib, sc)
    try:
        gpl = np.ascontiguousarray(plane, np.float32)
        mvs_lib.mvs_phi_select_min_cost(ctx.h, 0, known, h32, ovalid, c32, gpl)
    finally:
        ctx.close()
    f = ofilled.astype(bool)
    assert f.sum() > 500
    assert np.array_equal((gpl[..., 3] > 0) & (known == 0), f)
    assert np.array_equal(gpl[..., 3][f], opl[..., 3][f].astype(np.float32))
    assert np.abs(gpl[..., :3][f] - opl[..., :3][f]).max() <= 1e-3
    assert np.array_equal(gpl[known == 1], plane[known == 1].astype(np.float32))


def test_plane_infer_min_cost_end_to_end_parity(mvs_lib, oracle_lib):
    """The whole mvs_plane_infer in PHI-MVS/M mode against the oracle's from
    the same depth map: the hypothesis costs differ by rounding (FP32 against
    FP64), so choices may flip where two costs nearly tie."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=3, seed=41, baseline_frac=0.1, n_textured=2, n_flat=2,
                           flat_frac=0.2)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=3, seed=4)
    ctx = _ctx(mvs_lib, sc)
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    try:
        pl = np.zeros((120, 160, 4), np.float32)
        co = np.zeros((120, 160), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2, 3], p, pl, co)
        known = ((pl[..., 3] > 0) & (co < 0.5)).astype(np.uint8)
        opl, aux = oracle_lib.plane_infer(osc, 0, [1, 2, 3], p, known, pl.astype(np.float64), min_cost=True)
        gpl, gco = pl.copy(), co.copy()
        q = mvs_lib.PhiParams(selection=mvs_lib.MVS_PHI_SELECT_MIN_COST)
        mvs_lib.mvs_plane_infer(ctx.h, 0, [1, 2, 3], p, q, None, gpl, gco)
    finally:
        ctx.close()
    filled_o = aux["filled"].astype(bool)
    filled_g = (gpl[..., 3] > 0) & (known == 0)
    assert filled_o.sum() > 500
    assert (filled_o != filled_g).mean() < 0.01
    both = filled_o & filled_g
    # costs within the parity tolerance pick the same hypothesis outside near ties
    agree = np.abs(gpl[..., 3] - opl[..., 3]) <= 1e-3 * opl[..., 3]
    assert agree[both].mean() > 0.97
    assert np.array_equal(gpl[known == 1], pl[known == 1])


def test_table1_patchmatch_vs_phi_m_vs_phi(mvs_lib):
    """Table I analogue: completeness (depth within 1 % of the truth) of
    PatchMatch alone (PHI-MVS/P), with PHI selecting by minimal cost
    (PHI-MVS/M) and with the MRF (PHI-MVS).  Both PHI variants fill the
    texture-less regions PatchMatch cannot score."""
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=256, H=192, n_src=4, seed=31, baseline_frac=0.1, n_textured=2, n_flat=2,
                           flat_frac=0.25)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=4, seed=9)
    gt = sc.gt_depth
    flat = ~sc.gt_textured
    ctx = _ctx(mvs_lib, sc)
    try:
        pl = np.zeros((192, 256, 4), np.float32)
        co = np.zeros((192, 256), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2, 3, 4], p, pl, co)
        res = {"P": (np.abs(pl[..., 3] - gt) / gt < 0.01) & (co < 0.5)}
        for name, sel in (("M", mvs_lib.MVS_PHI_SELECT_MIN_COST), ("full", mvs_lib.MVS_PHI_SELECT_MRF)):
            a, b = pl.copy(), co.copy()
            mvs_lib.mvs_plane_infer(ctx.h, 0, [1, 2, 3, 4], p, mvs_lib.PhiParams(selection=sel), None, a, b)
            res[name] = np.abs(a[..., 3] - gt) / gt < 0.01     # (each call starts from the map it is given)
    finally:
        ctx.close()
    print({k: (round(float(v.mean()), 3), round(float(v[flat].mean()), 3)) for k, v in res.items()})
    # measured on this scene: all pixels 0.776 / 0.806 / 0.818, texture-less
    # 0.177 / 0.315 / 0.372 for P / M / full
    for k in ("M", "full"):
        assert res[k][flat].mean() > res["P"][flat].mean() + 0.1
        assert res[k].mean() > res["P"].mean() + 0.02
    # the paper's finding: choosing by the MRF beats choosing by cost alone
    assert res["full"][flat].mean() > res["M"][flat].mean()


def test_unknown_selection_is_rejected(mvs_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=32, H=24, n_src=2, seed=1)
    p = mvs_lib.PMParams(win_radius=5.0, win_samples=6, iters=1, seed=3)
    ctx = _ctx(mvs_lib, sc)
    try:
        pl = np.zeros((24, 32, 4), np.float32)
        co = np.zeros((24, 32), np.float32)
        mvs_lib.mvs_patchmatch(ctx.h, 0, [1, 2], p, pl, co)
        with pytest.raises(mvs_lib.MvsError) as e:
            mvs_lib.mvs_plane_infer(ctx.h, 0, [1, 2], p, mvs_lib.PhiParams(selection=2), None, pl, co)
        assert e.value.status == mvs_lib.MVS_EINVAL
    finally:
        ctx.close()
