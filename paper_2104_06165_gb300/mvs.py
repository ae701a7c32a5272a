"""Thin ctypes binding of libmvs.so (the C ABI declared in include/mvs.h).

Argument marshalling only: every step of the depth-map path runs in the
library's CUDA kernels.  Buffers may be torch CUDA tensors (device memory,
work is enqueued on the context's stream) or numpy arrays (host memory, the
call synchronises).  There is no CPU fallback: if the compiled library is
missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmvs.so")

MVS_OK, MVS_EINVAL, MVS_ENOMEM, MVS_ECUDA, MVS_ETIMEOUT, MVS_ESTATE, MVS_EUNSUPPORTED = range(7)
MVS_MEM_DEVICE, MVS_MEM_HOST = 0, 1
MVS_INIT_RANDOM, MVS_INIT_GIVEN, MVS_INIT_GIVEN_RECOST, MVS_INIT_RANGE = 0, 1, 2, 3
MVS_PHI_SELECT_MRF, MVS_PHI_SELECT_MIN_COST = 0, 1
(MVS_CNN_T_INPUT, MVS_CNN_T_ENC, MVS_CNN_T_POOL, MVS_CNN_T_CAT, MVS_CNN_T_DEC, MVS_CNN_T_HEAD, MVS_CNN_T_GRAD_HEAD,
 MVS_CNN_T_GRAD_DEC, MVS_CNN_T_GRAD_CAT, MVS_CNN_T_GRAD_ENC, MVS_CNN_T_GRAD_POOL) = range(11)
_CNN_ENC_CH = (32, 48, 64, 96, 128)
_CNN_DEC_CH = (32, 48, 64, 96)
_CNN_CAT_CH = (80, 112, 160, 224)
STATUS_NAMES = ["MVS_OK", "MVS_EINVAL", "MVS_ENOMEM", "MVS_ECUDA", "MVS_ETIMEOUT", "MVS_ESTATE",
                "MVS_EUNSUPPORTED"]


class MvsError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class mvs_camera(C.Structure):
    _fields_ = [("K", C.c_double * 9), ("R", C.c_double * 9), ("t", C.c_double * 3), ("width", C.c_int32),
                ("height", C.c_int32)]


class mvs_pm_params(C.Structure):
    _fields_ = [("win_radius", C.c_float), ("win_samples", C.c_int32), ("sigma_s", C.c_float),
                ("sigma_c", C.c_float), ("d_lo", C.c_float), ("d_hi", C.c_float), ("iters", C.c_int32),
                ("phase_begin", C.c_int32), ("phase_end", C.c_int32), ("init_mode", C.c_int32),
                ("seed", C.c_uint64), ("precision", C.c_int32), ("lanes_per_pixel", C.c_int32),
                ("n_prop", C.c_int32), ("reserved0", C.c_int32), ("proposals", C.c_void_p),
                ("init_range", C.c_void_p)]


class mvs_depth_map(C.Structure):
    _fields_ = [("plane", C.c_void_p), ("cost", C.c_void_p), ("mem", C.c_int32)]


class mvs_filter_params(C.Structure):
    _fields_ = [("depth_tol", C.c_float), ("depth_relative", C.c_int32), ("max_angle_deg", C.c_float),
                ("max_reproj_px", C.c_float), ("min_consistent", C.c_int32)]


class mvs_phi_params(C.Structure):
    _fields_ = [("kappa1", C.c_float), ("kappa2", C.c_float), ("kappa3", C.c_float), ("n_fit", C.c_int32),
                ("fit_inverse", C.c_int32), ("trw_iters", C.c_int32), ("hole_cost", C.c_float),
                ("selection", C.c_int32)]


@dataclass
class PMParams:
    """PatchMatch parameters; defaults follow Sec. IV (r_now = 5, r_orig = 7,
    8 iterations) with the bilateral weights sigma_s = 5 px, sigma_c = 0.2."""
    win_radius: float = 7.0
    win_samples: int = 11
    sigma_s: float = 5.0
    sigma_c: float = 0.2
    d_lo: float = 2.0
    d_hi: float = 8.0
    iters: int = 8
    phase_begin: int = 0
    phase_end: int = -1
    init_mode: int = MVS_INIT_RANDOM
    seed: int = 0
    precision: int = 0
    lanes_per_pixel: int = 0
    n_prop: int = 0
    proposals: object = None        # device buffer (H, W, n_prop, 4) float32 or None
    init_range: object = None       # device buffer (H, W, 2) float32 for MVS_INIT_RANGE, or None

    def c(self):
        pp = _ptr(self.proposals)[0] if self.proposals is not None else None
        rr = _ptr(self.init_range)[0] if self.init_range is not None else None
        return mvs_pm_params(self.win_radius, self.win_samples, self.sigma_s, self.sigma_c, self.d_lo, self.d_hi,
                             self.iters, self.phase_begin, self.phase_end, self.init_mode,
                             int(self.seed) & 0xFFFFFFFFFFFFFFFF, self.precision, self.lanes_per_pixel,
                             self.n_prop, 0, pp, rr)


@dataclass
class FilterParams:
    """Sec. III-D: 0.02 depth, 30 degrees, 1 px, more than one view."""
    depth_tol: float = 0.02
    depth_relative: int = 0
    max_angle_deg: float = 30.0
    max_reproj_px: float = 1.0
    min_consistent: int = 2

    def c(self):
        return mvs_filter_params(self.depth_tol, self.depth_relative, self.max_angle_deg, self.max_reproj_px,
                                 self.min_consistent)


@dataclass
class PhiParams:
    """Sec. III-E / Sec. IV: kappa = (4, 0.5, 2), six closest pixels, one
    TRW iteration."""
    kappa1: float = 4.0
    kappa2: float = 0.5
    kappa3: float = 2.0
    n_fit: int = 6
    fit_inverse: int = 0
    trw_iters: int = 1
    hole_cost: float = 0.5
    selection: int = 0          # MVS_PHI_SELECT_MRF; MVS_PHI_SELECT_MIN_COST = PHI-MVS/M

    def c(self):
        return mvs_phi_params(self.kappa1, self.kappa2, self.kappa3, self.n_fit, self.fit_inverse, self.trw_iters,
                              self.hole_cost, self.selection)


_lib = None


def load():
    """Load libmvs.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    vp, i32, ip, u8p, fp = C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p
    L.mvs_create.restype = i32
    L.mvs_create.argtypes = [C.POINTER(mvs_camera), C.POINTER(C.c_void_p), i32, vp, C.POINTER(C.c_void_p)]
    L.mvs_destroy.restype = None
    L.mvs_destroy.argtypes = [vp]
    L.mvs_last_error.restype = C.c_char_p
    L.mvs_last_error.argtypes = [vp]
    L.mvs_patchmatch.restype = i32
    L.mvs_patchmatch.argtypes = [vp, i32, ip, i32, C.POINTER(mvs_pm_params), C.POINTER(mvs_depth_map)]
    L.mvs_patchmatch_batch.restype = i32
    L.mvs_patchmatch_batch.argtypes = [vp, i32, ip, ip, i32, C.POINTER(mvs_pm_params), C.POINTER(mvs_depth_map)]
    L.mvs_plane_cost.restype = i32
    L.mvs_plane_cost.argtypes = [vp, i32, ip, i32, C.POINTER(mvs_pm_params), fp, fp, fp, i32]
    L.mvs_geo_filter.restype = i32
    L.mvs_geo_filter.argtypes = [vp, i32, ip, i32, C.POINTER(mvs_filter_params), u8p, vp, i32]
    L.mvs_plane_infer.restype = i32
    L.mvs_plane_infer.argtypes = [vp, i32, ip, i32, C.POINTER(mvs_pm_params), C.POINTER(mvs_phi_params), u8p,
                                  C.POINTER(mvs_depth_map)]
    L.mvs_phi_hypotheses.restype = i32
    L.mvs_phi_hypotheses.argtypes = [vp, i32, i32, fp, u8p, C.POINTER(mvs_phi_params), C.c_float, C.c_float, fp,
                                     u8p, i32]
    L.mvs_phi_hypotheses_static.restype = i32
    L.mvs_phi_hypotheses_static.argtypes = [vp, i32, i32, fp, u8p, C.POINTER(mvs_phi_params), C.c_float,
                                            C.c_float, fp, u8p]
    L.mvs_phi_cost.restype = i32
    L.mvs_phi_cost.argtypes = [vp, i32, ip, i32, C.POINTER(mvs_pm_params), fp, u8p, fp, i32]
    L.mvs_phi_mrf.restype = i32
    L.mvs_phi_mrf.argtypes = [vp, i32, i32, u8p, fp, fp, u8p, fp, C.POINTER(mvs_phi_params), vp, i32]
    L.mvs_phi_select.restype = i32
    L.mvs_phi_select.argtypes = [vp, i32, u8p, fp, u8p, vp, fp, i32]
    L.mvs_phi_select_min_cost.restype = i32
    L.mvs_phi_select_min_cost.argtypes = [vp, i32, u8p, fp, u8p, fp, fp, i32]
    L.mvs_profile.restype = i32
    L.mvs_profile.argtypes = [vp, i32]
    L.mvs_cnn_create.restype = i32
    L.mvs_cnn_create.argtypes = [i32, i32, C.c_float, C.c_float, C.c_uint64, vp, C.POINTER(C.c_void_p)]
    L.mvs_cnn_destroy.restype = None
    L.mvs_cnn_destroy.argtypes = [vp]
    L.mvs_cnn_last_error.restype = C.c_char_p
    L.mvs_cnn_last_error.argtypes = [vp]
    L.mvs_cnn_n_params.restype = i32
    L.mvs_cnn_n_params.argtypes = [vp, C.POINTER(C.c_int64)]
    for name in ("mvs_cnn_get_params", "mvs_cnn_set_params", "mvs_cnn_get_grads"):
        getattr(L, name).restype = i32
        getattr(L, name).argtypes = [vp, fp]
    L.mvs_cnn_forward.restype = i32
    L.mvs_cnn_forward.argtypes = [vp, u8p, fp, fp, i32, i32, fp]
    L.mvs_cnn_backward.restype = i32
    L.mvs_cnn_backward.argtypes = [vp, u8p, fp, fp, i32, i32, fp, u8p, C.POINTER(C.c_float)]
    L.mvs_set_depth_map.restype = i32
    L.mvs_set_depth_map.argtypes = [vp, i32, vp, vp, i32]
    L.mvs_measure_peaks.restype = i32
    L.mvs_measure_peaks.argtypes = [i32, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.mvs_cnn_test_timeout.restype = i32
    L.mvs_cnn_test_timeout.argtypes = [vp]
    L.mvs_cnn_read.restype = i32
    L.mvs_cnn_read.argtypes = [vp, i32, i32, vp, C.c_int64]
    L.mvs_cnn_adam_step.restype = i32
    L.mvs_cnn_adam_step.argtypes = [vp, C.c_float]
    L.mvs_cnn_propose.restype = i32
    L.mvs_cnn_propose.argtypes = [vp, u8p, fp, fp, i32, i32, C.POINTER(C.c_double), fp]
    L.mvs_propose.restype = i32
    L.mvs_propose.argtypes = [vp, i32, vp, fp]
    L.mvs_fuse.restype = i32
    L.mvs_fuse.argtypes = [vp, i32, ip, C.c_void_p, C.c_float, fp, vp, vp, C.c_int64, C.POINTER(C.c_int64), i32]
    L.mvs_select_neighbors.restype = i32
    L.mvs_select_neighbors.argtypes = [vp, C.c_int64, vp, vp, C.c_double, C.c_double, i32, vp, vp, vp, vp, i32]
    L.mvs_sparse_depth_range.restype = i32
    L.mvs_sparse_depth_range.argtypes = [vp, i32, C.c_int64, vp, vp, vp, vp, C.c_double, C.c_float, C.c_float, vp, i32]
    L.mvs_profile_read.restype = i32
    L.mvs_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]
    _lib = L
    return L


def _check(status, ctx=None):
    if status != MVS_OK:
        msg = load().mvs_last_error(ctx)
        raise MvsError(status, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, mem kind) of a torch CUDA tensor or a numpy array."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("numpy buffers must be C-contiguous")
        return a.ctypes.data, MVS_MEM_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor buffers must be contiguous")
        return a.data_ptr(), (MVS_MEM_DEVICE if a.is_cuda else MVS_MEM_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _mem(*bufs):
    kinds = {k for _, k in (_ptr(b) for b in bufs if b is not None)}
    if len(kinds) != 1:
        raise ValueError("all buffers of one call must be in the same memory (all device or all host)")
    return kinds.pop()


def _srcs(srcs):
    a = (C.c_int32 * len(srcs))(*[int(s) for s in srcs])
    return a, len(srcs)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def mvs_create(cams, images, stream=None):
    """cams: list of (K, R, t) with x_cam = R X + t; images: uint8 (H, W)
    numpy arrays.  Returns the context handle."""
    L = load()
    n = len(images)
    carr = (mvs_camera * n)()
    keep = []
    ptrs = (C.c_void_p * n)()
    for i, ((K, R, t), im) in enumerate(zip(cams, images)):
        im = np.ascontiguousarray(im, dtype=np.uint8)
        keep.append(im)
        carr[i].K[:] = [float(v) for v in np.asarray(K, float).ravel()]
        carr[i].R[:] = [float(v) for v in np.asarray(R, float).ravel()]
        carr[i].t[:] = [float(v) for v in np.asarray(t, float).ravel()]
        carr[i].height, carr[i].width = im.shape
        ptrs[i] = im.ctypes.data
    h = C.c_void_p()
    _check(L.mvs_create(carr, ptrs, n, _stream_handle(stream), C.byref(h)), None)
    return h


def mvs_destroy(ctx):
    load().mvs_destroy(ctx)


def mvs_patchmatch(ctx, ref, srcs, params: PMParams, plane, cost):
    """Run PatchMatch for view `ref`; plane (H, W, 4) float32 and cost (H, W)
    float32 buffers receive the result (and carry the start state for
    MVS_INIT_GIVEN*)."""
    pp, _ = _ptr(plane)
    cp, _ = _ptr(cost)
    mem = _mem(plane, cost)
    s, ns = _srcs(srcs)
    out = mvs_depth_map(pp, cp, mem)
    cpar = params.c()
    _check(load().mvs_patchmatch(ctx, ref, s, ns, C.byref(cpar), C.byref(out)), ctx)


def mvs_patchmatch_batch(ctx, refs, srcs, params: PMParams, planes, costs):
    """PatchMatch of several reference views in one captured CUDA graph.
    srcs: list of equal-length source lists, one per reference; planes /
    costs: per-reference buffers (all device or all host)."""
    n = len(refs)
    assert len(srcs) == n and len(planes) == n and len(costs) == n
    ns = len(srcs[0])
    assert all(len(s) == ns for s in srcs)
    mem = _mem(*planes, *costs)
    r = (C.c_int32 * n)(*[int(v) for v in refs])
    s = (C.c_int32 * (n * ns))(*[int(v) for row in srcs for v in row])
    outs = (mvs_depth_map * n)(*[mvs_depth_map(_ptr(pl)[0], _ptr(co)[0], mem) for pl, co in zip(planes, costs)])
    cpar = params.c()
    _check(load().mvs_patchmatch_batch(ctx, n, r, s, ns, C.byref(cpar), outs), ctx)


def mvs_plane_cost(ctx, ref, srcs, params: PMParams, plane, cost, view_cost=None):
    mem = _mem(plane, cost, view_cost)
    s, ns = _srcs(srcs)
    cpar = params.c()
    _check(load().mvs_plane_cost(ctx, ref, s, ns, C.byref(cpar), _ptr(plane)[0], _ptr(cost)[0],
                                 _ptr(view_cost)[0], mem), ctx)


def mvs_set_depth_map(ctx, view, plane, cost=None):
    """Store a depth map computed elsewhere (plane (H, W, 4), cost (H, W) or
    None) as view's state in the context."""
    mem = _mem(plane, cost)
    _check(load().mvs_set_depth_map(ctx, int(view), _ptr(plane)[0], _ptr(cost)[0], mem), ctx)


def mvs_geo_filter(ctx, ref, srcs, fparams: FilterParams, keep, count=None):
    mem = _mem(keep, count)
    s, ns = _srcs(srcs)
    cpar = fparams.c()
    _check(load().mvs_geo_filter(ctx, ref, s, ns, C.byref(cpar), _ptr(keep)[0], _ptr(count)[0], mem), ctx)


def mvs_fuse(ctx, views, points, src=None, keep_masks=None, rel_tol=0.01, owner=None):
    """Depth-map fusion of the context's maps of ``views`` (in that order)
    into ``points`` (capacity x 4 float32: x, y, z, merged count) and
    optionally ``src`` (capacity x 2 int32: view, pixel); ``keep_masks`` is
    None or one uint8 (H, W) mask or None per view; ``owner`` (optional,
    int64, one entry per pixel of the views in processing order) receives
    the index of the point each pixel went into, -1 if never present.
    Returns the number of points."""
    kms = list(keep_masks) if keep_masks is not None else []
    mem = _mem(points, src, owner, *[k for k in kms if k is not None])
    v, nv = _srcs(views)
    km = None
    if keep_masks is not None:
        if len(kms) != nv:
            raise ValueError("one keep mask (or None) per view")
        km = (C.c_void_p * nv)(*[_ptr(k)[0] for k in kms])
    cap = points.shape[0]
    n = C.c_int64(0)
    _check(load().mvs_fuse(ctx, nv, v, km, C.c_float(rel_tol), _ptr(points)[0], _ptr(src)[0], _ptr(owner)[0], cap,
                           C.byref(n), mem), ctx)
    return n.value


def mvs_select_neighbors(ctx, points, vis, neighbors, tau=None, n_shared=None, zeta=None, eps=0.002, t_tau=0.1):
    """Neighbouring-image selection of every context view from sparse points
    (n, 3) float64 and visibility masks vis (n,) uint64 (bit v: visible in
    view v) into neighbors (n_views, k) int32; optional (n_views, n_views)
    outputs tau / zeta (float64) and n_shared (int32).  eps and t_tau default
    to the values of Sec. IV (0.002, 0.1 px)."""
    mem = _mem(points, vis, neighbors, tau, n_shared, zeta)
    k = neighbors.shape[1]
    _check(load().mvs_select_neighbors(ctx, points.shape[0], _ptr(points)[0], _ptr(vis)[0], float(eps), float(t_tau),
                                       k, _ptr(neighbors)[0], _ptr(tau)[0], _ptr(n_shared)[0], _ptr(zeta)[0], mem),
           ctx)


def mvs_sparse_depth_range(ctx, ref, points, vis, reproj, obs, rng, max_reproj=2.0, d_lo=2.0, d_hi=8.0):
    """Per-pixel (d_min, d_max) of the sparse-feature initialisation of view
    ref into rng (H, W, 2) float32: points (n, 3) float64, vis (n,) uint64
    masks, reproj (n,) float64, obs (n, 2) float64 observations in ref."""
    mem = _mem(points, vis, reproj, obs, rng)
    _check(load().mvs_sparse_depth_range(ctx, ref, points.shape[0], _ptr(points)[0], _ptr(vis)[0], _ptr(reproj)[0],
                                         _ptr(obs)[0], float(max_reproj), C.c_float(d_lo), C.c_float(d_hi),
                                         _ptr(rng)[0], mem), ctx)


def mvs_plane_infer(ctx, ref, srcs, pm: PMParams, phi: PhiParams, keep_mask, plane, cost):
    mem = _mem(plane, cost, keep_mask)
    s, ns = _srcs(srcs)
    out = mvs_depth_map(_ptr(plane)[0], _ptr(cost)[0], mem)
    a, b = pm.c(), phi.c()
    _check(load().mvs_plane_infer(ctx, ref, s, ns, C.byref(a), C.byref(b), _ptr(keep_mask)[0], C.byref(out)), ctx)


def mvs_phi_hypotheses(ctx, depth, known, phi: PhiParams, d_lo, d_hi, hyp, valid):
    mem = _mem(depth, known, hyp, valid)
    H, W = depth.shape
    b = phi.c()
    _check(load().mvs_phi_hypotheses(ctx, W, H, _ptr(depth)[0], _ptr(known)[0], C.byref(b), d_lo, d_hi,
                                     _ptr(hyp)[0], _ptr(valid)[0], mem), ctx)


def mvs_phi_hypotheses_static(ctx, depth, known, phi: PhiParams, d_lo, d_hi, hyp, valid):
    """mvs_phi_hypotheses without any device allocation (device buffers only;
    at most MVS_PHI_STATIC_MAX_PIXELS pixels)."""
    if _mem(depth, known, hyp, valid) != MVS_MEM_DEVICE:
        raise ValueError("mvs_phi_hypotheses_static takes device buffers only")
    H, W = depth.shape
    b = phi.c()
    _check(load().mvs_phi_hypotheses_static(ctx, W, H, _ptr(depth)[0], _ptr(known)[0], C.byref(b), d_lo, d_hi,
                                            _ptr(hyp)[0], _ptr(valid)[0]), ctx)


MVS_PHI_STATIC_MAX_PIXELS = 262144


def mvs_phi_cost(ctx, ref, srcs, pm: PMParams, hyp, valid, hcost):
    mem = _mem(hyp, valid, hcost)
    s, ns = _srcs(srcs)
    a = pm.c()
    _check(load().mvs_phi_cost(ctx, ref, s, ns, C.byref(a), _ptr(hyp)[0], _ptr(valid)[0], _ptr(hcost)[0], mem),
           ctx)


def mvs_phi_mrf(ctx, known, depth, hyp, valid, hcost, phi: PhiParams, label):
    mem = _mem(known, depth, hyp, valid, hcost, label)
    H, W = depth.shape
    b = phi.c()
    _check(load().mvs_phi_mrf(ctx, W, H, _ptr(known)[0], _ptr(depth)[0], _ptr(hyp)[0], _ptr(valid)[0],
                              _ptr(hcost)[0], C.byref(b), _ptr(label)[0], mem), ctx)


def mvs_phi_select(ctx, ref, known, hyp, valid, label, plane):
    mem = _mem(known, hyp, valid, label, plane)
    _check(load().mvs_phi_select(ctx, ref, _ptr(known)[0], _ptr(hyp)[0], _ptr(valid)[0], _ptr(label)[0],
                                 _ptr(plane)[0], mem), ctx)


def mvs_phi_select_min_cost(ctx, ref, known, hyp, valid, hcost, plane):
    mem = _mem(known, hyp, valid, hcost, plane)
    _check(load().mvs_phi_select_min_cost(ctx, ref, _ptr(known)[0], _ptr(hyp)[0], _ptr(valid)[0], _ptr(hcost)[0],
                                          _ptr(plane)[0], mem), ctx)


def mvs_measure_peaks(device=0):
    """(FP32 flop/s, L1 gathers/s, L2 read bytes/s) measured on `device`."""
    f, g, b = C.c_double(), C.c_double(), C.c_double()
    st = load().mvs_measure_peaks(int(device), C.byref(f), C.byref(g), C.byref(b))
    if st != MVS_OK:
        raise MvsError(st, "mvs_measure_peaks failed")
    return f.value, g.value, b.value


def mvs_profile(ctx, enable):
    _check(load().mvs_profile(ctx, int(bool(enable))), ctx)


def mvs_profile_read(ctx):
    """(phase kernel ms, phase launches, kernel launches, ZNCC evaluations)"""
    ms = C.c_double()
    a, b, e = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().mvs_profile_read(ctx, C.byref(ms), C.byref(a), C.byref(b), C.byref(e)), ctx)
    return ms.value, a.value, b.value, e.value


def _check_cnn(status, net):
    if status != MVS_OK:
        msg = load().mvs_cnn_last_error(net)
        raise MvsError(status, msg.decode() if msg else "")


def _dev(*bufs):
    for b in bufs:
        if _ptr(b)[1] != MVS_MEM_DEVICE:
            raise ValueError("the proposal network takes device buffers only")
    return [_ptr(b)[0] for b in bufs]


def mvs_cnn_create(max_width, max_height, d_lo, d_hi, seed=0, stream=None):
    h = C.c_void_p()
    _check_cnn(load().mvs_cnn_create(int(max_width), int(max_height), float(d_lo), float(d_hi),
                                     int(seed) & 0xFFFFFFFFFFFFFFFF, _stream_handle(stream), C.byref(h)), None)
    return h


def mvs_cnn_destroy(net):
    load().mvs_cnn_destroy(net)


def mvs_cnn_n_params(net):
    n = C.c_int64()
    _check_cnn(load().mvs_cnn_n_params(net, C.byref(n)), net)
    return n.value


def mvs_cnn_get_params(net):
    a = np.zeros(mvs_cnn_n_params(net), np.float32)
    _check_cnn(load().mvs_cnn_get_params(net, a.ctypes.data), net)
    return a


def mvs_cnn_set_params(net, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != mvs_cnn_n_params(net):
        raise ValueError("parameter count mismatch")
    _check_cnn(load().mvs_cnn_set_params(net, a.ctypes.data), net)


def mvs_cnn_get_grads(net):
    a = np.zeros(mvs_cnn_n_params(net), np.float32)
    _check_cnn(load().mvs_cnn_get_grads(net, a.ctypes.data), net)
    return a


def mvs_cnn_test_timeout(net):
    """Runs the bounded-wait check of the convolutions; returns the status
    code (MVS_ETIMEOUT expected) without raising."""
    return load().mvs_cnn_test_timeout(net)


def mvs_cnn_read(net, tensor, level, W, H):
    """A stored tensor of the last forward / backward pass at size W x H:
    (H >> l, W >> l, channels) float32 (bf16 values widened exactly)."""
    ch = {MVS_CNN_T_INPUT: 16, MVS_CNN_T_HEAD: 16, MVS_CNN_T_GRAD_HEAD: 16}.get(tensor)
    lv = level
    if tensor in (MVS_CNN_T_ENC, MVS_CNN_T_GRAD_ENC):
        ch = _CNN_ENC_CH[level]
    elif tensor in (MVS_CNN_T_POOL, MVS_CNN_T_GRAD_POOL):
        ch, lv = _CNN_ENC_CH[level], level + 1
    elif tensor in (MVS_CNN_T_CAT, MVS_CNN_T_GRAD_CAT):
        ch = _CNN_CAT_CH[level]
    elif tensor in (MVS_CNN_T_DEC, MVS_CNN_T_GRAD_DEC):
        ch = _CNN_DEC_CH[level]
    shape = (H >> lv, W >> lv, ch)
    if tensor == MVS_CNN_T_HEAD:
        a = np.zeros(shape, np.float32)
        _check_cnn(load().mvs_cnn_read(net, tensor, level, a.ctypes.data, a.nbytes), net)
        return a
    a = np.zeros(shape, np.uint16)
    _check_cnn(load().mvs_cnn_read(net, tensor, level, a.ctypes.data, a.nbytes), net)
    return (a.astype(np.uint32) << 16).view(np.float32)


def mvs_cnn_forward(net, img, plane, cost, out):
    """img (H, W) uint8, plane (H, W, 4), cost (H, W) -> out (H, W, 16)."""
    H, W = img.shape
    pi, pp, pc, po = _dev(img, plane, cost, out)
    _check_cnn(load().mvs_cnn_forward(net, pi, pp, pc, W, H, po), net)


def mvs_cnn_backward(net, img, plane, cost, target, mask):
    """Forward + loss against target planes on mask + backward; returns the loss."""
    H, W = img.shape
    pi, pp, pc, pt, pm = _dev(img, plane, cost, target, mask)
    loss = C.c_float()
    _check_cnn(load().mvs_cnn_backward(net, pi, pp, pc, W, H, pt, pm, C.byref(loss)), net)
    return loss.value


def mvs_cnn_adam_step(net, lr):
    _check_cnn(load().mvs_cnn_adam_step(net, float(lr)), net)


def mvs_cnn_propose(net, img, plane, cost, Kinv, proposals):
    H, W = img.shape
    pi, pp, pc, pr = _dev(img, plane, cost, proposals)
    k = (C.c_double * 9)(*[float(v) for v in np.asarray(Kinv, float).ravel()])
    _check_cnn(load().mvs_cnn_propose(net, pi, pp, pc, W, H, k, pr), net)


def mvs_propose(ctx, ref, net, proposals):
    """Proposals (H, W, 4, 4) float32 device buffer from the current map of `ref`."""
    (pr,) = _dev(proposals)
    _check(load().mvs_propose(ctx, int(ref), net, pr), ctx)


class Context:
    """Owns an mvs_ctx for a scene (cameras + uint8 images)."""

    def __init__(self, K, R, t, images, stream=None):
        cams = [(K[i], R[i], t[i]) for i in range(len(images))]
        self.h = mvs_create(cams, images, stream)
        self.shapes = [np.asarray(im).shape for im in images]

    def close(self):
        if self.h is not None and self.h.value:
            mvs_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
