"""Seeded synthetic multi-view scenes (input generator only).

Stands in for the ETH3D high-resolution scenes of the paper's experiments
(Sec. IV), which are not available here.  A scene is a set of planar quads
(one large background plane, textured quads and texture-less quads) seen by
one reference camera and several source cameras.  Images are rendered by
ray casting in double precision; textures are band-limited sums of
sinusoids in plane coordinates; intensities are mapped to [20, 235] and
rounded half-to-even to uint8.  Ground-truth depth (z-depth) and normals of
the reference view come with the render.

This module holds no arithmetic of the depth-estimation method itself; it
feeds both the CUDA library and the CPU oracle with the same arrays.
Random numbers of the method are drawn inside the method (Philox); the seeds
here only shape the scene.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Quad:
    center: np.ndarray        # world point
    normal: np.ndarray        # unit world normal
    e1: np.ndarray            # in-plane unit axes
    e2: np.ndarray
    half: tuple               # half extents along e1, e2
    textured: bool
    flat_value: float = 128.0
    freqs: np.ndarray = None  # (K, 2) cycles per world unit
    phases: np.ndarray = None
    amps: np.ndarray = None
    blanks: list = field(default_factory=list)   # texture-less patches: (c1, c2, h1, h2, value) in plane coords


@dataclass
class Scene:
    K: np.ndarray             # (n, 3, 3)
    R: np.ndarray             # (n, 3, 3) world -> camera
    t: np.ndarray             # (n, 3)
    images: list              # uint8 (H, W) per view (or float64 in [0,1])
    gt_depth: np.ndarray      # reference view z-depth (H, W), 0 = nothing hit
    gt_normal: np.ndarray     # reference view normals (H, W, 3), facing the camera
    gt_textured: np.ndarray   # bool (H, W): reference pixel lies on a textured quad
    d_lo: float
    d_hi: float
    quads: list = field(default_factory=list)

    @property
    def n_views(self):
        return len(self.images)


def intrinsics(W, H, f):
    return np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])


def look_at(C, target, down=(0.0, 1.0, 0.0)):
    """Rotation (world -> camera, rows = camera axes x right, y down, z
    forward) and translation of a camera at C looking at target."""
    C = np.asarray(C, float)
    z = np.asarray(target, float) - C
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(down, float), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return R, -R @ C


def _plane_axes(n):
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(n, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return e1, e2


def _texture(rng, depth, f, n_sin=32, lam_px=(4.0, 32.0), std=38.0):
    """Band-limited texture: n_sin sinusoids with wavelengths log-uniform in
    lam_px pixels at the given depth."""
    lam = np.exp(rng.uniform(np.log(lam_px[0]), np.log(lam_px[1]), n_sin)) * depth / f
    ang = rng.uniform(0, np.pi, n_sin)
    freqs = np.stack([np.cos(ang), np.sin(ang)], 1) / lam[:, None]
    phases = rng.uniform(0, 2 * np.pi, n_sin)
    amps = rng.uniform(0.5, 1.0, n_sin)
    amps *= std / math.sqrt(0.5 * np.sum(amps ** 2))
    return freqs, phases, amps


def _random_normal(rng, max_tilt_deg):
    """Unit normal facing the reference camera (negative z), tilted up to
    max_tilt_deg from the optical axis."""
    tilt = math.radians(rng.uniform(0, max_tilt_deg))
    az = rng.uniform(0, 2 * math.pi)
    return np.array([math.sin(tilt) * math.cos(az), math.sin(tilt) * math.sin(az), -math.cos(tilt)])


def _ray_dirs(K, R, W, H, y0, y1):
    v, u = np.mgrid[y0:y1, 0:W].astype(np.float64)
    pix = np.stack([u, v, np.ones_like(u)], -1)
    d_cam = pix @ np.linalg.inv(K).T
    return d_cam @ R  # world directions (rows): R^T d


def _render_rows(quads, K, R, t, W, H, y0, y1, want_gt):
    C = -R.T @ t
    dirs = _ray_dirs(K, R, W, H, y0, y1)
    best = np.full(dirs.shape[:2], np.inf)
    idx = np.full(dirs.shape[:2], -1, np.int32)
    for qi, q in enumerate(quads):
        den = dirs @ q.normal
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = ((q.center - C) @ q.normal) / den
        P = C + lam[..., None] * dirs
        rel = P - q.center
        s1, s2 = rel @ q.e1, rel @ q.e2
        hit = (lam > 1e-9) & (np.abs(s1) <= q.half[0]) & (np.abs(s2) <= q.half[1]) & (lam < best)
        best = np.where(hit, lam, best)
        idx = np.where(hit, qi, idx)
    img = np.full(dirs.shape[:2], 128.0)
    for qi, q in enumerate(quads):
        m = idx == qi
        if not m.any():
            continue
        if not q.textured:
            img[m] = q.flat_value
            continue
        P = C + best[m][:, None] * dirs[m]
        rel = P - q.center
        s1, s2 = rel @ q.e1, rel @ q.e2
        acc = np.zeros(s1.shape)
        for k in range(len(q.amps)):
            acc += q.amps[k] * np.sin(2 * np.pi * (q.freqs[k, 0] * s1 + q.freqs[k, 1] * s2) + q.phases[k])
        val = 128.0 + acc
        for (c1, c2, h1, h2, bv) in q.blanks:
            val = np.where((np.abs(s1 - c1) <= h1) & (np.abs(s2 - c2) <= h2), bv, val)
        img[m] = val
    out = {"img": img}
    if want_gt:
        P = C + np.where(np.isfinite(best), best, 0.0)[..., None] * dirs
        Pc = P @ R.T + t
        depth = np.where(idx >= 0, Pc[..., 2], 0.0)
        nrm = np.zeros(dirs.shape[:2] + (3,))
        tex = np.zeros(dirs.shape[:2], bool)
        for qi, q in enumerate(quads):
            m = idx == qi
            nc = R @ q.normal
            nrm[m] = nc
            tex[m] = q.textured
            if q.textured and q.blanks and m.any():
                P = C + best[m][:, None] * dirs[m]
                rel = P - q.center
                s1, s2 = rel @ q.e1, rel @ q.e2
                t_ = np.ones(s1.shape, bool)
                for (c1, c2, h1, h2, bv) in q.blanks:
                    t_ &= ~((np.abs(s1 - c1) <= h1) & (np.abs(s2 - c2) <= h2))
                tex[m] = t_
        ray_c = np.stack(np.meshgrid(np.arange(W, dtype=float), np.arange(y0, y1, dtype=float)), -1)
        ray_c = np.concatenate([ray_c, np.ones(ray_c.shape[:2] + (1,))], -1) @ np.linalg.inv(K).T
        flip = np.sum(nrm * ray_c, -1) > 0
        nrm[flip] *= -1
        out.update(depth=depth, normal=nrm, textured=tex)
    return out


def render(quads, K, R, t, W, H, quantise=True, want_gt=False, threads=None):
    if threads is None:
        threads = 1 if W * H < 500_000 else min(16, os.cpu_count() or 1)
    step = max(8, (H + threads * 4 - 1) // (threads * 4))
    chunks = [(y, min(H, y + step)) for y in range(0, H, step)]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda c: _render_rows(quads, K, R, t, W, H, c[0], c[1], want_gt), chunks))
    img = np.concatenate([p["img"] for p in parts], 0)
    if quantise:
        img = np.rint(np.clip(img, 20.0, 235.0)).astype(np.uint8)
    else:
        img = np.clip(img, 20.0, 235.0) / 255.0
    out = {"img": img}
    if want_gt:
        for k in ("depth", "normal", "textured"):
            out[k] = np.concatenate([p[k] for p in parts], 0)
    return out


def _quad_facing(rng, K, W, H, depth, u, v, size_px, textured, f, tilt=50.0, flat_value=None, tex_std=38.0):
    """Quad whose centre projects to reference pixel (u, v) at the given
    depth, roughly size_px pixels across, tilted up to `tilt` degrees."""
    ray = np.linalg.inv(K) @ np.array([u, v, 1.0])
    center = depth * ray
    n = _random_normal(rng, tilt)
    e1, e2 = _plane_axes(n)
    half = size_px * depth / f / 2.0
    q = Quad(center=center, normal=n, e1=e1, e2=e2, half=(half, half * rng.uniform(0.6, 1.0)),
             textured=textured)
    if textured:
        q.freqs, q.phases, q.amps = _texture(rng, depth, f, std=tex_std)
    else:
        q.flat_value = float(flat_value if flat_value is not None else rng.uniform(70, 190))
    return q


def _sources_ring(n_src, z_c, angles_deg, rng):
    """Source camera centres at the given viewing angles to the scene
    centre (0, 0, z_c), azimuths spread around the reference axis."""
    cams = []
    for k in range(n_src):
        a = math.radians(angles_deg[k])
        b = 2 * math.pi * k / n_src + rng.uniform(-0.2, 0.2)
        C = np.array([0.0, 0.0, z_c]) + z_c * np.array([math.sin(a) * math.cos(b), math.sin(a) * math.sin(b),
                                                        -math.cos(a)])
        cams.append(look_at(C, [0.0, 0.0, z_c]))
    return cams


def make_scene(W=320, H=240, f=None, n_src=4, seed=0, baseline_frac=0.1, view_angles=None,
               n_textured=3, n_flat=1, flat_frac=None, d_lo=2.0, d_hi=8.0, quantise=True, threads=None,
               flat_bg=0.0, tex_std=38.0, noise_std=0.0):
    """Scene of textured planar quads in front of a textured background plane,
    with n_flat texture-less (constant-intensity) patches painted on those
    planes.

    Default shape: W x H reference, focal f = 300 * W / 320 px (same field of
    view at every resolution), n_src source views.  With view_angles=None the
    sources sit on a ring of radius baseline_frac * 5 around the reference
    optical axis; otherwise at the given viewing angles (degrees) to the
    scene centre.  flat_frac sizes the patches so that roughly that fraction
    of the reference image is texture-less (default 8 %); flat_bg > 0 adds
    three blank squares on the background plane at random image positions,
    together about that fraction of the image before occlusion.  tex_std is
    the texture contrast (grey levels); noise_std > 0 adds independent
    Gaussian noise of that deviation to every view before rounding."""
    rng = np.random.default_rng(seed)
    f = f if f is not None else 300.0 * W / 320.0
    K = intrinsics(W, H, f)
    z_c = 5.0
    quads = []
    # background: large textured plane at depth ~7, mildly tilted
    bg_depth = 7.0
    n_bg = _random_normal(rng, 15.0)
    e1, e2 = _plane_axes(n_bg)
    bg = Quad(center=np.array([0.0, 0.0, bg_depth]), normal=n_bg, e1=e1, e2=e2, half=(40.0, 40.0), textured=True)
    bg.freqs, bg.phases, bg.amps = _texture(rng, bg_depth, f, std=tex_std)
    quads.append(bg)
    placed = []
    for k in range(n_textured):
        for _ in range(50):
            u = rng.uniform(0.15 * W, 0.85 * W)
            v = rng.uniform(0.15 * H, 0.85 * H)
            if all((u - pu) ** 2 + (v - pv) ** 2 > (0.18 * W) ** 2 for pu, pv in placed):
                break
        placed.append((u, v))
        depth = rng.uniform(3.0, 5.8)
        size = rng.uniform(0.3, 0.45) * W
        quads.append(_quad_facing(rng, K, W, H, depth, u, v, size, True, f, tilt=50.0, tex_std=tex_std))
    # texture-less regions: blank patches painted on the textured quads, each
    # centred on its quad and sized for flat_frac of the reference image in
    # total (at most 80 % of the quad's side), so that a blank region is
    # surrounded by texture of its own plane
    target = (flat_frac if flat_frac is not None else 0.08) * W * H / max(n_flat, 1)
    for k in range(n_flat):
        q = quads[1 + k % max(n_textured, 1)] if n_textured else quads[0]
        pc = K @ q.center
        depth_c = pc[2]
        quad_px = (2 * q.half[0] * f / depth_c) * (2 * q.half[1] * f / depth_c)
        side = float(np.clip(math.sqrt(target / quad_px), 0.2, 0.8))
        c1, c2 = rng.uniform(-0.1, 0.1) * q.half[0], rng.uniform(-0.1, 0.1) * q.half[1]
        q.blanks.append((c1, c2, side * q.half[0], side * q.half[1], float(rng.uniform(70, 190))))
    if flat_bg > 0:
        Kinv = np.linalg.inv(K)
        side_px = math.sqrt(flat_bg * W * H / 3.0)
        for k in range(3):
            u, v = rng.uniform(0.1 * W, 0.9 * W), rng.uniform(0.1 * H, 0.9 * H)
            r = Kinv @ np.array([u, v, 1.0])
            X = r * (bg.normal @ bg.center) / (bg.normal @ r)
            half = 0.5 * side_px * X[2] / f
            bg.blanks.append((float(bg.e1 @ (X - bg.center)), float(bg.e2 @ (X - bg.center)), half, half,
                              float(rng.uniform(70, 190))))
    Ks, Rs, ts = [K], [np.eye(3)], [np.zeros(3)]
    if view_angles is None:
        b = baseline_frac * z_c
        for k in range(n_src):
            a = 2 * math.pi * k / n_src
            R, t = look_at([b * math.cos(a), b * math.sin(a), 0.0], [0.0, 0.0, z_c])
            Ks.append(K); Rs.append(R); ts.append(t)
    else:
        for R, t in _sources_ring(n_src, z_c, view_angles, rng):
            Ks.append(K); Rs.append(R); ts.append(t)
    images = []
    gt = None
    for v in range(len(Ks)):
        out = render(quads, Ks[v], Rs[v], ts[v], W, H, quantise=quantise and noise_std <= 0, want_gt=(v == 0),
                     threads=threads)
        img = out["img"]
        if noise_std > 0:     # render gave [0, 1] floats: noise in grey levels
            img = img * 255.0 + rng.normal(0.0, noise_std, img.shape)
            img = np.clip(np.rint(img), 0, 255).astype(np.uint8) if quantise else np.clip(img, 0, 255) / 255.0
        images.append(img)
        if v == 0:
            gt = out
    return Scene(K=np.stack(Ks), R=np.stack(Rs), t=np.stack(ts), images=images, gt_depth=gt["depth"],
                 gt_normal=gt["normal"], gt_textured=gt["textured"], d_lo=d_lo, d_hi=d_hi, quads=quads)


def make_plane_scene(W=64, H=48, f=None, n_src=2, seed=0, depth=4.0, normal=(0.0, 0.0, -1.0),
                     baseline=0.2, quantise=True, textured=True, flat_value=128.0, lam_px=(4.0, 16.0)):
    """A single infinite-extent textured plane through (0, 0, depth) with the
    given world normal, sources translated along x (and y) from the
    reference without rotation."""
    rng = np.random.default_rng(seed)
    f = f if f is not None else 300.0 * W / 320.0
    K = intrinsics(W, H, f)
    n = np.asarray(normal, float)
    n /= np.linalg.norm(n)
    e1, e2 = _plane_axes(n)
    q = Quad(center=np.array([0.0, 0.0, depth]), normal=n, e1=e1, e2=e2, half=(1e3, 1e3), textured=textured,
             flat_value=flat_value)
    if textured:
        q.freqs, q.phases, q.amps = _texture(rng, depth, f, lam_px=lam_px)
    Ks, Rs, ts = [K], [np.eye(3)], [np.zeros(3)]
    for k in range(n_src):
        a = 2 * math.pi * k / n_src
        C = np.array([baseline * math.cos(a), baseline * math.sin(a), 0.0])
        Ks.append(K); Rs.append(np.eye(3)); ts.append(-C)
    images, gt = [], None
    for v in range(len(Ks)):
        out = render([q], Ks[v], Rs[v], ts[v], W, H, quantise=quantise, want_gt=(v == 0), threads=1)
        images.append(out["img"])
        if v == 0:
            gt = out
    return Scene(K=np.stack(Ks), R=np.stack(Rs), t=np.stack(ts), images=images, gt_depth=gt["depth"],
                 gt_normal=gt["normal"], gt_textured=gt["textured"], d_lo=2.0, d_hi=8.0, quads=[q])


# ---------------------------------------------------------------------------
# Workload shapes (stand-ins for the paper's ETH3D high-resolution inputs)
# ---------------------------------------------------------------------------
def scene_small(seed=0, **kw):
    """320 x 240, 4 sources at baseline 0.1 x scene depth, 3 textured quads in
    front of a textured background, one texture-less patch, depth [2, 8]."""
    return make_scene(W=320, H=240, n_src=4, seed=seed, baseline_frac=0.1, n_textured=3, n_flat=1, **kw)


def scene_highres(seed=0, W=3072, H=2048, n_src=10, **kw):
    """3072 x 2048 reference + 10 sources at 15..40 degree viewing angles,
    texture-less patches sized for about 30 % of the reference."""
    angles = list(np.linspace(15.0, 40.0, n_src))
    return make_scene(W=W, H=H, n_src=n_src, seed=seed, view_angles=angles, n_textured=4, n_flat=4,
                      flat_frac=0.30, **kw)


def scene_batch(seed=0, sizes=((3072, 2048),) * 8 + ((2048, 1365),) * 8 + ((1536, 1024),) * 8, n_src=10,
                n_textured=4, n_flat=4, flat_frac=0.25, want_gt=False, threads=None):
    """Many reference views of one scene at mixed resolutions (focal length
    scaled with the width: same field of view).  Cameras sit on three rings
    around the axis through the scene centre (0, 0, 5), every one looking at
    it; each view's sources are the n_src others whose viewing directions
    differ from its own by the angle closest to 25 degrees (within 15..40
    degrees where possible).  Returns (Scene with per-view images, list of
    source lists)."""
    rng = np.random.default_rng(seed)
    W0, H0 = sizes[0]
    f0 = 300.0 * W0 / 320.0
    K0 = intrinsics(W0, H0, f0)
    # geometry framed for the first camera, as in make_scene
    base = make_scene(W=64, H=int(round(64 * H0 / W0)), n_src=0, seed=seed, n_textured=n_textured, n_flat=n_flat,
                      flat_frac=flat_frac)
    quads = base.quads
    z_c = 5.0
    n = len(sizes)
    dirs = []
    rings = [(6.0, n // 3), (20.0, n // 3), (34.0, n - 2 * (n // 3))]
    for ri, (alpha, cnt) in enumerate(rings):
        for k in range(cnt):
            beta = 2 * math.pi * (k + 0.5 * ri) / cnt + rng.uniform(-0.05, 0.05)
            a = math.radians(alpha)
            dirs.append(np.array([math.sin(a) * math.cos(beta), math.sin(a) * math.sin(beta), -math.cos(a)]))
    Ks, Rs, ts, images, gts = [], [], [], [], []
    for v in range(n):
        W, H = sizes[v]
        f = 300.0 * W / 320.0
        K = intrinsics(W, H, f)
        C = np.array([0.0, 0.0, z_c]) + z_c * dirs[v]
        R, t = look_at(C, [0.0, 0.0, z_c])
        out = render(quads, K, R, t, W, H, quantise=True, want_gt=want_gt, threads=threads)
        Ks.append(K); Rs.append(R); ts.append(t); images.append(out["img"])
        gts.append(out if want_gt else None)
    srcs = []
    for v in range(n):
        ang = [math.degrees(math.acos(float(np.clip(dirs[v] @ dirs[u], -1, 1)))) if u != v else 1e9
               for u in range(n)]
        order = sorted(range(n), key=lambda u: (0 if 15.0 <= ang[u] <= 40.0 else 1, abs(ang[u] - 25.0)))
        srcs.append([u for u in order if u != v][:n_src])
    g0 = gts[0]
    sc = Scene(K=np.stack(Ks), R=np.stack(Rs), t=np.stack(ts), images=images,
               gt_depth=g0["depth"] if g0 else None, gt_normal=g0["normal"] if g0 else None,
               gt_textured=g0["textured"] if g0 else None, d_lo=2.0, d_hi=8.0, quads=quads)
    sc.gt_views = gts
    return sc, srcs


def sparse_points(sc, n_points=4000, seed=0, obs_noise_px=0.5, outlier_frac=0.02):
    """Synthetic structure-from-motion output for a scene: 3D points on the
    textured parts of the quads (features are found on texture), each the
    surface point seen through a uniformly drawn pixel of a random view, their visibility in every view (in front, inside the image and
    not occluded by another quad), an observation per visible view (the
    projection plus Gaussian noise of obs_noise_px) and the mean
    reprojection error of the stored point.  A fraction outlier_frac of the
    points is stored displaced by 2..10 % of its distance to the first
    camera (wrong reconstructions, with large reprojection errors).

    Returns dict(X (N, 3), vis (N, n_views) bool, obs (N, n_views, 2) with
    NaN where not visible, reproj (N,))."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n_points:
        # the surface point seen through a random pixel of a random view
        v = int(rng.integers(sc.n_views))
        H, W = sc.images[v].shape
        u, w = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        C = -sc.R[v].T @ sc.t[v]
        d = sc.R[v].T @ (np.linalg.inv(sc.K[v]) @ np.array([u, w, 1.0]))
        best, hit = np.inf, None
        for Q in sc.quads:
            den = d @ Q.normal
            if abs(den) < 1e-12:
                continue
            s_ = ((Q.center - C) @ Q.normal) / den
            P = C + s_ * d - Q.center
            a, b = P @ Q.e1, P @ Q.e2
            if 0 < s_ < best and abs(a) <= Q.half[0] and abs(b) <= Q.half[1]:
                best, hit = s_, (Q, a, b)
        if hit is None:
            continue
        Q, a, b = hit
        if not Q.textured or any(abs(a - c1) <= h1 and abs(b - c2) <= h2 for (c1, c2, h1, h2, _) in Q.blanks):
            continue
        pts.append(C + best * d)
    X = np.array(pts)
    n = sc.n_views
    vis = np.zeros((len(X), n), bool)
    obs = np.full((len(X), n, 2), np.nan)
    for v in range(n):
        K, R, t = sc.K[v], sc.R[v], sc.t[v]
        H, W = sc.images[v].shape
        C = -R.T @ t
        q = (X @ R.T + t) @ K.T
        z = q[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u, w = q[:, 0] / z, q[:, 1] / z
        ok = (z > 0) & (u >= 0) & (u <= W - 1) & (w >= 0) & (w <= H - 1)
        # occlusion: does the segment from the camera centre to X cross a quad?
        d = X - C
        for Q in sc.quads:
            den = d @ Q.normal
            with np.errstate(divide="ignore", invalid="ignore"):
                s = ((Q.center - C) @ Q.normal) / den
            P = C + s[:, None] * d - Q.center
            hit = (s > 1e-9) & (s < 1.0 - 1e-6) & (np.abs(P @ Q.e1) <= Q.half[0]) & (np.abs(P @ Q.e2) <= Q.half[1])
            ok &= ~hit
        vis[:, v] = ok
        obs[ok, v, 0] = u[ok] + rng.normal(0, obs_noise_px, ok.sum())
        obs[ok, v, 1] = w[ok] + rng.normal(0, obs_noise_px, ok.sum())
    # wrong reconstructions: the stored point moves off the surface
    bad = rng.uniform(size=len(X)) < outlier_frac
    C0 = -sc.R[0].T @ sc.t[0]
    dirs = rng.normal(size=(len(X), 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    X = X + bad[:, None] * dirs * np.linalg.norm(X - C0, axis=1, keepdims=True) * rng.uniform(0.02, 0.10, (len(X), 1))
    rep = np.zeros(len(X))
    for v in range(n):
        q = (X @ sc.R[v].T + sc.t[v]) @ sc.K[v].T
        with np.errstate(divide="ignore", invalid="ignore"):
            e = np.hypot(q[:, 0] / q[:, 2] - obs[:, v, 0], q[:, 1] / q[:, 2] - obs[:, v, 1])
        rep += np.where(vis[:, v], e, 0.0)
    rep /= np.maximum(vis.sum(1), 1)
    return dict(X=X, vis=vis, obs=obs, reproj=rep)
