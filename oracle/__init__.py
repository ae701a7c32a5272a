"""FP64 CPU oracle of the PHI-MVS depth-map path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2104_06165_gb300``) never imports it and has no CPU
fallback.

The arithmetic lives in ``mvs_oracle.c`` (plain C, double precision, single
thread); this module builds it with gcc and marshals numpy arrays through
ctypes.  Each wrapper names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mvs_oracle.c")
_LIB = os.path.join(_HERE, "libmvs_oracle.so")
_lock = threading.Lock()
_lib = None

CMAX = 2.0  # C_max = 1 - Z_min with Z_min = -1 (Sec. III-C)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no FMA contraction so
    x86-64 and aarch64 hosts give the same double-precision results)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _PM(C.Structure):
    _fields_ = [("win_radius", C.c_double), ("win_samples", C.c_int), ("sigma_s", C.c_double),
                ("sigma_c", C.c_double), ("d_lo", C.c_double), ("d_hi", C.c_double),
                ("seed", C.c_uint64), ("n_prop", C.c_int), ("props", C.POINTER(C.c_double)),
                ("init_range", C.POINTER(C.c_float))]


class _Filter(C.Structure):
    _fields_ = [("depth_tol", C.c_double), ("depth_relative", C.c_int), ("max_angle_deg", C.c_double),
                ("max_reproj", C.c_double), ("min_consistent", C.c_int)]


class _Phi(C.Structure):
    _fields_ = [("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double), ("n_fit", C.c_int),
                ("inverse", C.c_int), ("trw_iters", C.c_int), ("min_cost", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp, ip, up = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_uint8)
            vp = C.c_void_p
            L.or_scene_create.restype = vp
            L.or_scene_create.argtypes = [C.c_int, dp, dp, dp, ip, ip, C.POINTER(dp)]
            L.or_scene_destroy.argtypes = [vp]
            L.or_philox4x64.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
            L.or_bilinear.restype = C.c_double
            L.or_bilinear.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double]
            L.or_window_offsets.argtypes = [C.POINTER(_PM), dp]
            L.or_homography.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_double, dp]
            L.or_plane_cost.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_PM), dp, dp, dp, dp]
            L.or_window_extent.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_PM), dp, dp]
            L.or_wzncc.restype = C.c_double
            L.or_wzncc.argtypes = [C.c_int, dp, dp, dp]
            L.or_aggregate.restype = C.c_double
            L.or_aggregate.argtypes = [C.c_int, dp, ip]
            L.or_init.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_PM), dp, dp]
            L.or_group_members.restype = C.c_int
            L.or_group_members.argtypes = [C.c_int, ip]
            L.or_phase.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_PM), C.c_int, dp, dp, ip, dp, ip, dp, dp]
            L.or_patchmatch.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_PM), C.c_int, dp, dp]
            L.or_geo_filter.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_Filter), C.POINTER(dp), up, ip, dp]
            L.or_phi_hypotheses.argtypes = [C.c_int, C.c_int, dp, up, C.c_int, C.c_int, C.c_double, C.c_double,
                                            dp, up]
            L.or_line_fit_at.restype = C.c_double
            L.or_line_fit_at.argtypes = [dp, up, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                         C.c_double, C.c_double, ip]
            L.or_phi_cost.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_PM), dp, up, dp, dp]
            L.or_phi_mrf.argtypes = [C.c_int, C.c_int, up, dp, dp, up, dp, C.c_double, C.c_double, C.c_double,
                                     C.c_int, ip, dp]
            L.or_phi_select.argtypes = [vp, C.c_int, up, dp, up, ip, dp, up, dp]
            L.or_phi_select_min_cost.argtypes = [vp, C.c_int, up, dp, up, dp, dp, up]
            L.or_phi_unary.restype = C.c_double
            L.or_phi_unary.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_phi_pair.restype = C.c_double
            L.or_phi_pair.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_trw.argtypes = [C.c_int, C.c_int, ip, dp, dp, C.c_double, C.c_int, dp, ip]
            L.or_mrf_energy.restype = C.c_double
            L.or_mrf_energy.argtypes = [C.c_int, C.c_int, ip, dp, dp, C.c_double, ip]
            L.or_eq10_normal.restype = C.c_int
            L.or_eq10_normal.argtypes = [vp, C.c_int, dp, C.c_int, C.c_int, dp]
            L.or_plane_infer.argtypes = [vp, C.c_int, ip, C.c_int, C.POINTER(_PM), C.POINTER(_Phi), up, dp,
                                         dp, up, dp, ip, dp, up]
            L.or_fuse.restype = C.c_long
            lp = C.POINTER(C.c_long)
            L.or_fuse.argtypes = [vp, C.c_int, ip, C.POINTER(dp), C.POINTER(up), C.c_double, C.c_double,
                                  C.c_double, lp, dp, ip, lp, lp, C.c_long, lp]
            L.or_select_neighbors.argtypes = [vp, C.c_long, dp, up, C.c_double, C.c_double, C.c_int, ip, dp, ip, dp]
            L.or_sparse_features.restype = C.c_long
            L.or_sparse_features.argtypes = [vp, C.c_int, C.c_long, dp, up, dp, dp, C.c_double, dp, dp]
            L.or_sparse_range.argtypes = [C.c_int, C.c_int, C.c_long, dp, dp, C.c_double, C.c_double, C.c_double,
                                          dp, up]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _u8(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _pm(p, props=None, init_range=None) -> _PM:
    """props: None or an FP64 array (H, W, K, 4); init_range: None or a
    float32 array (H, W, 2); both kept alive by the caller."""
    rng = init_range.ctypes.data_as(C.POINTER(C.c_float)) if init_range is not None else None
    if props is None:
        return _PM(float(p.win_radius), int(p.win_samples), float(p.sigma_s), float(p.sigma_c),
                   float(p.d_lo), float(p.d_hi), int(p.seed) & 0xFFFFFFFFFFFFFFFF, 0, None, rng)
    return _PM(float(p.win_radius), int(p.win_samples), float(p.sigma_s), float(p.sigma_c),
               float(p.d_lo), float(p.d_hi), int(p.seed) & 0xFFFFFFFFFFFFFFFF, int(props.shape[2]), _d(props), rng)


class Scene:
    """Cameras (K, R, t; x_cam = R X + t) and images of all views.

    ``images`` are uint8 (scaled by 1/255, reading of the intensity scale)
    or float arrays already in [0, 1] (unquantised renders for the exactness
    pins)."""

    def __init__(self, K, R, t, images):
        self.n = len(images)
        self.K = _f64(np.asarray(K).reshape(self.n, 9))
        self.R = _f64(np.asarray(R).reshape(self.n, 9))
        self.t = _f64(np.asarray(t).reshape(self.n, 3))
        imgs = []
        for im in images:
            im = np.asarray(im)
            imgs.append(_f64(im / 255.0) if im.dtype == np.uint8 else _f64(im))
        self.images = imgs
        self.W = np.array([im.shape[1] for im in imgs], dtype=np.int32)
        self.H = np.array([im.shape[0] for im in imgs], dtype=np.int32)
        ptrs = (C.POINTER(C.c_double) * self.n)(*[_d(im) for im in imgs])
        self._ptrs = ptrs
        self.h = lib().or_scene_create(self.n, _d(self.K), _d(self.R), _d(self.t), _i(self.W), _i(self.H), ptrs)

    def __del__(self):
        try:
            if getattr(self, "h", None) and _lib is not None:
                _lib.or_scene_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def shape(self, v):
        return int(self.H[v]), int(self.W[v])


def _srcs(srcs):
    return np.ascontiguousarray(srcs, dtype=np.int32)


def philox4x64(ctr, key):
    """Philox4x64-10 block (Salmon et al., SC'11)."""
    c = (C.c_uint64 * 4)(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in key])
    o = (C.c_uint64 * 4)()
    lib().or_philox4x64(c, k, o)
    return [int(o[i]) for i in range(4)]


def bilinear(img, u, v):
    im = _f64(img)
    return lib().or_bilinear(_d(im), im.shape[1], im.shape[0], float(u), float(v))


def window_offsets(p):
    out = np.zeros(int(p.win_samples), np.float64)
    lib().or_window_offsets(C.byref(_pm(p)), _d(out))
    return out


def homography(scene, ref, j, x, y, n, d):
    n = _f64(n)
    out = np.zeros(9, np.float64)
    lib().or_homography(scene.h, ref, j, x, y, _d(n), float(d), _d(out))
    return out.reshape(3, 3)


def plane_cost(scene, ref, srcs, p, plane, with_views=False):
    """Eq. 4/5 cost of a given plane map (H, W, 4) = (nx, ny, nz, depth).
    Returns cost (H, W), per-view costs (H, W, n_src) and the decision
    margin (H, W)."""
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    pl = _f64(plane).reshape(H, W, 4)
    cost = np.zeros((H, W), np.float64)
    vc = np.zeros((H, W, len(s)), np.float64)
    mg = np.zeros((H, W), np.float64)
    lib().or_plane_cost(scene.h, ref, _i(s), len(s), C.byref(_pm(p)), _d(pl), _d(cost), _d(vc), _d(mg))
    return (cost, vc, mg) if with_views else cost


def window_extent(scene, ref, srcs, p, plane):
    """Per pixel and source view, the extent (source pixels) of the window's
    image under the pixel's plane (a comparison diagnostic; see
    or_window_extent).  Returns (H, W, n_src)."""
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    pl = _f64(plane).reshape(H, W, 4)
    ext = np.zeros((H, W, len(s)), np.float64)
    lib().or_window_extent(scene.h, ref, _i(s), len(s), C.byref(_pm(p)), _d(pl), _d(ext))
    return ext


def cost_at(scene, ref, srcs, p, xs, ys, planes):
    """Eq. 4/5 cost (and decision margin) of planes (n, 4) at the reference
    pixels (xs[k], ys[k]) only."""
    s = _srcs(srcs)
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    pl = np.ascontiguousarray(_f64(planes).reshape(-1, 4))
    n = len(xs)
    cost = np.zeros(n, np.float64)
    mg = np.zeros(n, np.float64)
    lib().or_cost_at(scene.h, ref, _i(s), len(s), C.byref(_pm(p)), n, _i(xs), _i(ys), _d(pl), _d(cost), _d(mg))
    return cost, mg


def wzncc(w, a, b):
    w, a, b = _f64(w), _f64(a), _f64(b)
    return lib().or_wzncc(len(w), _d(w), _d(a), _d(b))


def aggregate(cj, ok):
    cj = _f64(cj)
    ok = np.ascontiguousarray(ok, dtype=np.int32)
    return lib().or_aggregate(len(cj), _d(cj), _i(ok))


def init(scene, ref, srcs, p, with_cost=True, init_range=None):
    """Sec. III-B random initialisation (Philox draws) and its cost;
    init_range (H, W, 2) float32 gives per-pixel depth ranges (NaN: none)."""
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    plane = np.zeros((H, W, 4), np.float64)
    cost = np.zeros((H, W), np.float64)
    rng = None if init_range is None else np.ascontiguousarray(init_range, np.float32)
    lib().or_init(scene.h, ref, _i(s), len(s), C.byref(_pm(p, init_range=rng)), _d(plane),
                  _d(cost) if with_cost else None)
    return plane, cost


def group_members(g):
    out = np.zeros(32, np.int32)
    c = lib().or_group_members(g, _i(out))
    return out[: 2 * c].reshape(c, 2)


def phase(scene, ref, srcs, p, ph, plane, cost, proposals=None):
    """One checkerboard half-iteration (propagation, learned proposals when
    given as an (H, W, K, 4) plane array, refinement) starting from the given
    state.  Returns the new (plane, cost) and a dict of decision diagnostics
    (win_prop is 8 + k when proposal k won)."""
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    props = None if proposals is None else np.ascontiguousarray(proposals, dtype=np.float64)
    pl = _f64(plane).reshape(H, W, 4).copy()
    co = _f64(cost).reshape(H, W).copy()
    wp = np.zeros((H, W), np.int32)
    wr = np.zeros((H, W), np.int32)
    gp = np.zeros((H, W), np.float64)
    gr = np.zeros((H, W), np.float64)
    mg = np.full((H, W), np.inf, np.float64)
    pm = _pm(p, props)
    lib().or_phase(scene.h, ref, _i(s), len(s), C.byref(pm), int(ph), _d(pl), _d(co), _i(wp), _d(gp),
                   _i(wr), _d(gr), _d(mg))
    return pl, co, {"win_prop": wp, "gap_prop": gp, "win_ref": wr, "gap_ref": gr, "margin": mg}


def patchmatch(scene, ref, srcs, p, iters):
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    plane = np.zeros((H, W, 4), np.float64)
    cost = np.zeros((H, W), np.float64)
    lib().or_patchmatch(scene.h, ref, _i(s), len(s), C.byref(_pm(p)), int(iters), _d(plane), _d(cost))
    return plane, cost


def geo_filter(scene, ref, srcs, planes, depth_tol=0.02, depth_relative=False, max_angle_deg=30.0,
               max_reproj=1.0, min_consistent=2, with_margin=False):
    """Sec. III-D geometric-consistency filter. ``planes`` maps view index
    to its (H, W, 4) plane map. Returns keep mask (uint8) and counts, and with
    ``with_margin`` also each pixel's decision margin (below 1: a float
    evaluation of the same tests may decide that pixel either way; the bands
    are stated in or_geo_filter)."""
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    arrs = [None] * scene.n
    for v, pl in planes.items():
        arrs[v] = _f64(pl)
    ptrs = (C.POINTER(C.c_double) * scene.n)(*[(_d(a) if a is not None else C.POINTER(C.c_double)())
                                               for a in arrs])
    keep = np.zeros((H, W), np.uint8)
    cnt = np.zeros((H, W), np.int32)
    f = _Filter(depth_tol, int(depth_relative), max_angle_deg, max_reproj, min_consistent)
    margin = np.zeros((H, W), np.float64)
    lib().or_geo_filter(scene.h, ref, _i(s), len(s), C.byref(f), ptrs, _u8(keep), _i(cnt), _d(margin))
    return (keep, cnt, margin) if with_margin else (keep, cnt)


def phi_hypotheses(depth, known, n_fit=6, inverse=False, d_lo=0.0, d_hi=np.inf):
    """Sec. III-E four-direction line-fit hypotheses."""
    depth = _f64(depth)
    known = np.ascontiguousarray(known, dtype=np.uint8)
    H, W = depth.shape
    hyp = np.zeros((H, W, 4), np.float64)
    valid = np.zeros((H, W, 4), np.uint8)
    lib().or_phi_hypotheses(W, H, _d(depth), _u8(known), n_fit, int(inverse), float(d_lo), float(d_hi),
                            _d(hyp), _u8(valid))
    return hyp, valid


def line_fit_at(depth, known, x, y, k, n_fit=6, inverse=False, d_lo=0.0, d_hi=np.inf):
    depth = _f64(depth)
    known = np.ascontiguousarray(known, dtype=np.uint8)
    H, W = depth.shape
    ok = C.c_int(0)
    h = lib().or_line_fit_at(_d(depth), _u8(known), W, H, x, y, k, n_fit, int(inverse), float(d_lo),
                             float(d_hi), C.byref(ok))
    return (h if ok.value else None)


def phi_cost(scene, ref, srcs, p, hyp, valid, with_margin=False):
    """Sec. III-E hypothesis costs (fronto-parallel plane at each depth)."""
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    hyp = _f64(hyp)
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    out = np.zeros((H, W, 4), np.float64)
    mg = np.zeros((H, W, 4), np.float64)
    lib().or_phi_cost(scene.h, ref, _i(s), len(s), C.byref(_pm(p)), _d(hyp), _u8(valid), _d(out), _d(mg))
    return (out, mg) if with_margin else out


def phi_mrf(known, depth, hyp, valid, hcost, k1=4.0, k2=0.5, k3=2.0, iters=1):
    """Sec. III-E MRF at half resolution from full-resolution inputs; returns
    labels (gh, gw) (-1 reconstructed node, -2 absent) and belief gaps."""
    known = np.ascontiguousarray(known, dtype=np.uint8)
    H, W = known.shape
    gw, gh = (W + 1) // 2, (H + 1) // 2
    label = np.zeros((gh, gw), np.int32)
    gap = np.zeros((gh, gw), np.float64)
    lib().or_phi_mrf(W, H, _u8(known), _d(_f64(depth)), _d(_f64(hyp)),
                     _u8(np.ascontiguousarray(valid, dtype=np.uint8)), _d(_f64(hcost)), k1, k2, k3, iters,
                     _i(label), _d(gap))
    return label, gap


def phi_select(scene, ref, known, hyp, valid, label, plane):
    """Sec. III-E selection + Eq. 10 normals; returns (plane, filled)."""
    H, W = scene.shape(ref)
    pl = _f64(plane).reshape(H, W, 4).copy()
    filled = np.zeros((H, W), np.uint8)
    refd = np.zeros((H, W), np.float64)
    lib().or_phi_select(scene.h, ref, _u8(np.ascontiguousarray(known, dtype=np.uint8)), _d(_f64(hyp)),
                        _u8(np.ascontiguousarray(valid, dtype=np.uint8)),
                        _i(np.ascontiguousarray(label, dtype=np.int32)), _d(pl), _u8(filled), _d(refd))
    return pl, filled


def phi_select_min_cost(scene, ref, known, hyp, valid, hcost, plane):
    """PHI-MVS/M selection (Sec. IV, Table I): each hole takes its valid
    hypothesis of minimal matching cost, then Eq. 10 normals; returns (plane,
    filled)."""
    H, W = scene.shape(ref)
    pl = _f64(plane).reshape(H, W, 4).copy()
    filled = np.zeros((H, W), np.uint8)
    lib().or_phi_select_min_cost(scene.h, ref, _u8(np.ascontiguousarray(known, np.uint8)), _d(_f64(hyp)),
                                 _u8(np.ascontiguousarray(valid, np.uint8)), _d(_f64(hcost)), _d(pl), _u8(filled))
    return pl, filled


def phi_unary(c, k1=4.0, k2=0.5):
    return lib().or_phi_unary(float(c), float(k1), float(k2))


def phi_pair(h1, h2, k3=2.0):
    return lib().or_phi_pair(float(h1), float(h2), float(k3))


def trw(nlab, lab, un, k3=2.0, iters=1):
    """TRW min-sum decoding on a grid (reading of Sec. III-E's TRW).
    nlab (gh, gw) int, lab/un (gh, gw, 4). Returns labels (gh, gw)
    (-1 for absent nodes) and the messages."""
    nlab = np.ascontiguousarray(nlab, dtype=np.int32)
    gh, gw = nlab.shape
    lab, un = _f64(lab), _f64(un)
    msg = np.zeros((gh, gw, 4, 4), np.float64)
    label = np.zeros((gh, gw), np.int32)
    lib().or_trw(gw, gh, _i(nlab), _d(lab), _d(un), float(k3), int(iters), _d(msg), _i(label))
    return label, msg


def mrf_energy(nlab, lab, un, label, k3=2.0):
    nlab = np.ascontiguousarray(nlab, dtype=np.int32)
    gh, gw = nlab.shape
    lab, un = _f64(lab), _f64(un)
    label = np.ascontiguousarray(label, dtype=np.int32)
    return lib().or_mrf_energy(gw, gh, _i(nlab), _d(lab), _d(un), float(k3), _i(label))


def eq10_normal(scene, ref, depth, x, y):
    depth = _f64(depth)
    n = np.zeros(3, np.float64)
    ok = lib().or_eq10_normal(scene.h, ref, _d(depth), x, y, _d(n))
    return n if ok else None


def plane_infer(scene, ref, srcs, p, known, plane, k1=4.0, k2=0.5, k3=2.0, n_fit=6, inverse=False,
                trw_iters=1, min_cost=False):
    """Sec. III-E: hypotheses, their costs, half-resolution MRF, selection,
    Eq. 10 normals (min_cost: PHI-MVS/M, the minimal-cost hypothesis per
    hole without the MRF).  Returns the filled plane map and the
    intermediates."""
    H, W = scene.shape(ref)
    s = _srcs(srcs)
    known = np.ascontiguousarray(known, dtype=np.uint8)
    pl = _f64(plane).reshape(H, W, 4).copy()
    gw, gh = (W + 1) // 2, (H + 1) // 2
    hyp = np.zeros((H, W, 4), np.float64)
    valid = np.zeros((H, W, 4), np.uint8)
    hcost = np.zeros((H, W, 4), np.float64)
    label = np.zeros((gh, gw), np.int32)
    refd = np.zeros((H, W), np.float64)
    filled = np.zeros((H, W), np.uint8)
    q = _Phi(k1, k2, k3, n_fit, int(inverse), trw_iters, int(bool(min_cost)))
    lib().or_plane_infer(scene.h, ref, _i(s), len(s), C.byref(_pm(p)), C.byref(q), _u8(known), _d(pl),
                         _d(hyp), _u8(valid), _d(hcost), _i(label), _d(refd), _u8(filled))
    return pl, {"hyp": hyp, "valid": valid, "hcost": hcost, "label": label, "refdepth": refd,
                "filled": filled}


def fuse(scene, order, planes, keep=None, rel_tol=0.01, hint=None, band_px=0.0, band_rel=0.0, stats=False):
    """Sec. III-F depth-map fusion of the views in ``order`` in FP64 (see
    or_fuse).  ``planes`` maps view index to its (H, W, 4) plane map,
    ``keep`` optionally to a uint8 mask.  ``hint``: another implementation's
    per-pixel point index (views in ``order`` back to back), followed only at
    decisions within ``band_px`` of a rounding boundary or ``band_rel`` (of
    the threshold) of the 1 % test.  Returns (points (n, 4) float64 = x, y,
    z, merged count; source view (n,); source pixel (n,)), plus the per-pixel
    owner array and the counts (projections, fragile, resolved by the hint)
    when ``stats``."""
    order = [int(v) for v in order]
    n = len(order)
    arrs = [_f64(planes[v]) for v in order]
    kps = [None if keep is None or keep.get(v) is None else np.ascontiguousarray(keep[v], np.uint8) for v in order]
    dps = (C.POINTER(C.c_double) * n)(*[_d(a) for a in arrs])
    ups = (C.POINTER(C.c_ubyte) * n)(*[(_u8(k) if k is not None else C.POINTER(C.c_ubyte)()) for k in kps])
    cap = int(sum(scene.shape(v)[0] * scene.shape(v)[1] for v in order))
    lp = lambda a: a.ctypes.data_as(C.POINTER(C.c_long))
    pts = np.zeros((max(cap, 1), 4), np.float64)
    sv = np.zeros(max(cap, 1), np.int32)
    sp = np.zeros(max(cap, 1), np.int64)
    own = np.zeros(max(cap, 1), np.int64)
    st = np.zeros(3, np.int64)
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, np.int64).ravel()
        if h.size != cap:
            raise ValueError("hint needs one entry per pixel of the views")
    m = lib().or_fuse(scene.h, n, _i(np.asarray(order, np.int32)), dps, ups, float(rel_tol), float(band_px),
                      float(band_rel), lp(h) if h is not None else C.POINTER(C.c_long)(), _d(pts), _i(sv), lp(sp),
                      lp(own), cap, lp(st))
    if stats:
        return pts[:m], sv[:m], sp[:m], own[:cap], {"projections": int(st[0]), "fragile": int(st[1]),
                                                    "resolved_by_hint": int(st[2])}
    return pts[:m], sv[:m], sp[:m]


def select_neighbors(scene, X, vis, eps=0.002, t_tau=0.1, k=8):
    """Sec. III-A neighbouring-image selection (Eqs. 1-3) from sparse points
    X (n, 3) and their visibility vis (n, n_views) bool; eps and t_tau
    default to Sec. IV's 0.002 and 0.1 px, k to the paper's eight.  Returns (neighbours
    (n_views, k) int, -1 padded; tau, n_shared, zeta (n_views, n_views))."""
    X = _f64(np.asarray(X).reshape(-1, 3))
    vis = np.ascontiguousarray(vis, np.uint8)
    n = scene.n
    nbr = np.zeros((n, k), np.int32)
    tau = np.zeros((n, n))
    na = np.zeros((n, n), np.int32)
    zeta = np.zeros((n, n))
    lib().or_select_neighbors(scene.h, len(X), _d(X), _u8(vis), float(eps), float(t_tau), int(k), _i(nbr), _d(tau),
                              _i(na), _d(zeta))
    return nbr, tau, na, zeta


def sparse_features(scene, ref, X, vis, reproj, obs, max_reproj=2.0):
    """Sec. III-B features of view ref from sparse points (X (n, 3), vis
    (n, n_views) bool, reproj (n,), obs (n, 2) observations in ref).
    Returns (uv (m, 2) float64, depth (m,) float64)."""
    X = _f64(np.asarray(X).reshape(-1, 3))
    vis = np.ascontiguousarray(vis, np.uint8)
    n = len(X)
    obs = _f64(np.nan_to_num(np.asarray(obs, np.float64).reshape(n, 2)))
    uv = np.zeros((max(n, 1), 2), np.float64)
    dep = np.zeros(max(n, 1), np.float64)
    m = lib().or_sparse_features(scene.h, ref, n, _d(X), _u8(vis), _d(_f64(reproj)), _d(obs), float(max_reproj),
                                 _d(uv), _d(dep))
    return uv[:m], dep[:m]


def sparse_range(W, H, uv, depth, d_lo=2.0, d_hi=8.0, band_px=0.0, fragile=False):
    """Per-pixel (d_min, d_max) of the closest features in four quadrants
    within W / 10 px (NaN: none), (H, W, 2) float64; with ``fragile`` also
    the (H, W) mask of pixels whose choice lies within ``band_px`` of a
    boundary."""
    uv = _f64(np.asarray(uv, np.float64).reshape(-1, 2))
    depth = _f64(np.asarray(depth, np.float64).ravel())
    out = np.zeros((H, W, 2), np.float64)
    fr = np.zeros((H, W), np.uint8)
    lib().or_sparse_range(int(W), int(H), len(depth), _d(uv), _d(depth), float(d_lo), float(d_hi), float(band_px),
                          _d(out), _u8(fr))
    return (out, fr.astype(bool)) if fragile else out
