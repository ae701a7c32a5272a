"""Neighbouring-image selection (Sec. III-A) on the GPU against the FP64
oracle, on synthetic structure-from-motion points of rendered scenes, with
Sec. IV's eps = 0.002 and t_tau = 0.1 px (the defaults of both sides)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _masks(vis):
    m = np.zeros(len(vis), np.uint64)
    for v in range(vis.shape[1]):
        m |= vis[:, v].astype(np.uint64) << np.uint64(v)
    return m


def _compare(mvs_lib, oracle_lib, sc, sp, k):
    import torch
    n = sc.n_views
    ctx = mvs_lib.Context(sc.K, sc.R, sc.t, sc.images, stream=torch.cuda.current_stream())
    try:
        X = np.ascontiguousarray(sp["X"], np.float64)
        m = _masks(sp["vis"])
        nbr = np.zeros((n, k), np.int32)
        tau = np.zeros((n, n))
        na = np.zeros((n, n), np.int32)
        zeta = np.zeros((n, n))
        mvs_lib.mvs_select_neighbors(ctx.h, X, m, nbr, tau, na, zeta)
        # device buffers give the same selection
        d_nbr = torch.zeros((n, k), dtype=torch.int32, device="cuda")
        mvs_lib.mvs_select_neighbors(ctx.h, torch.from_numpy(X).cuda(), torch.from_numpy(m.view(np.int64)).cuda(),
                                     d_nbr)
        assert np.array_equal(d_nbr.cpu().numpy(), nbr)
    finally:
        ctx.close()
    osc = oracle_lib.Scene(sc.K, sc.R, sc.t, sc.images)
    onbr, otau, ona, ozeta = oracle_lib.select_neighbors(osc, sp["X"], sp["vis"], k=k)
    assert np.array_equal(na, ona)
    assert np.allclose(tau, otau, rtol=1e-12, atol=0)
    # no source sits within rounding of the threshold, so the removals are unique
    off = ~np.eye(n, dtype=bool)
    assert (np.abs(otau[off] - 0.1) > 1e-9).all()
    assert np.array_equal(np.isinf(zeta), np.isinf(ozeta))
    fin = np.isfinite(ozeta)
    assert np.allclose(zeta[fin], ozeta[fin], rtol=1e-12, atol=0)
    assert np.array_equal(nbr, onbr)
    return nbr, otau


def test_selection_equals_oracle_on_a_ring(mvs_lib, oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=6, seed=3, view_angles=[2.0, 8.0, 15.0, 25.0, 35.0, 50.0])
    sp = scenes.sparse_points(sc, 3000, seed=1)
    nbr, tau = _compare(mvs_lib, oracle_lib, sc, sp, k=4)
    # at this image size (f = 150 px) the sources at 2, 8 and 15 degrees move
    # projections by less than t_tau = 0.1 px: removed
    assert (tau[0, 1:4] < 0.1).all() and not {1, 2, 3} & set(nbr[0].tolist())
    assert nbr[0].tolist() == [5, 6, 4, -1]


def test_selection_equals_oracle_on_many_views(mvs_lib, oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc, _ = scenes.scene_batch(seed=2, sizes=((192, 128),) * 24)
    sp = scenes.sparse_points(sc, 6000, seed=4)
    nbr, _ = _compare(mvs_lib, oracle_lib, sc, sp, k=8)
    assert (nbr >= 0).all()


def test_short_lists_are_padded(mvs_lib, oracle_lib):
    from paper_2104_06165_gb300 import scenes
    sc = scenes.make_scene(W=160, H=120, n_src=6, seed=3, view_angles=[2.0, 8.0, 15.0, 25.0, 35.0, 50.0])
    sp = scenes.sparse_points(sc, 3000, seed=1)
    nbr, _ = _compare(mvs_lib, oracle_lib, sc, sp, k=6)
    assert (nbr[0, 3:] == -1).all()      # three of the six sources fall below t_tau
