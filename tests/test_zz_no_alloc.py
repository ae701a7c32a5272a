"""The allocation-free entry point mvs_phi_hypotheses_static.

Callers that cannot allocate device memory at run time (a fixed memory
budget reserved at start-up, an engine that owns every device byte, or a
pipeline that cannot take the device-wide synchronisation of cudaMalloc)
use this variant; it keeps its scratch in a fixed array inside the library.
Its results must equal those of mvs_phi_hypotheses, call after call.

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(rng, H, W):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    depth = 3.0 + 0.01 * xx + 0.02 * yy + 0.3 * np.sin(xx / 7.0) * np.cos(yy / 5.0)
    known = (rng.uniform(size=(H, W)) > 0.35).astype(np.uint8)
    known[H // 4: H // 2, W // 3: 2 * W // 3] = 0
    return (depth * known).astype(np.float32), known


def test_static_scratch_variant_matches_allocating_entry_point(mvs_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=32, H=24, n_src=1, seed=0)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    rng = np.random.default_rng(42)
    phi = mvs_lib.PhiParams()
    try:
        # two calls in a row, different sizes and contents
        for (H, W) in [(96, 160), (211, 173)]:
            depth, known = _inputs(rng, H, W)
            d = torch.from_numpy(depth).cuda()
            k = torch.from_numpy(known).cuda()
            hyp_a = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
            val_a = torch.zeros((H, W, 4), dtype=torch.uint8, device="cuda")
            hyp_b = torch.full((H, W, 4), -1.0, dtype=torch.float32, device="cuda")
            val_b = torch.full((H, W, 4), 7, dtype=torch.uint8, device="cuda")
            mvs_lib.mvs_phi_hypotheses(ctx.h, d, k, phi, 2.0, 8.0, hyp_a, val_a)
            mvs_lib.mvs_phi_hypotheses_static(ctx.h, d, k, phi, 2.0, 8.0, hyp_b, val_b)
            torch.cuda.synchronize()
            va, vb = val_a.cpu().numpy(), val_b.cpu().numpy()
            ha, hb = hyp_a.cpu().numpy(), hyp_b.cpu().numpy()
            assert np.array_equal(va, vb)
            assert va.sum() > 1000
            both = va == 1
            # same kernels, same inputs: equal within the PHI tests' tolerance (in fact bit for bit)
            assert np.abs(ha[both] - hb[both]).max() <= 1e-4 * np.abs(ha[both]).max()
            assert np.array_equal(ha, hb)
    finally:
        ctx.close()


def test_static_scratch_variant_rejects_oversized_input(mvs_lib):
    import torch
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_plane_scene(W=32, H=24, n_src=1, seed=0)
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    try:
        H, W = 600, 500          # 300,000 pixels > 262,144
        assert H * W > mvs_lib.MVS_PHI_STATIC_MAX_PIXELS
        d = torch.zeros((H, W), dtype=torch.float32, device="cuda")
        k = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        hyp = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
        val = torch.zeros((H, W, 4), dtype=torch.uint8, device="cuda")
        with pytest.raises(mvs_lib.MvsError) as e:
            mvs_lib.mvs_phi_hypotheses_static(ctx.h, d, k, mvs_lib.PhiParams(), 2.0, 8.0, hyp, val)
        assert e.value.status == mvs_lib.MVS_EINVAL and "exceeds" in str(e.value)
    finally:
        ctx.close()
