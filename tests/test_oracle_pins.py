"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
a library routine, brute force, an invariant or finite differences.  Equation
references are to RT-GuIDE (arXiv 2409.18122), Sec. III "Gaussian Splatting"
(projection and compositing) and Eq. (2) (mapping by back-propagation).
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2409_18122_gb300.scenes import Camera, GaussianMap, random_scene

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def gmap_from(mu, ls, q, logit, rgb, u):
    n = len(mu)
    mo = np.zeros((n, 4), np.float32)
    mo[:, :3] = mu
    mo[:, 3] = logit
    su = np.zeros((n, 4), np.float32)
    su[:, :3] = ls
    su[:, 3] = u
    c = np.zeros((n, 4), np.float32)
    c[:, :3] = rgb
    return GaussianMap(mo, su, np.asarray(q, np.float32), c)


def sig(x):
    return 1.0 / (1.0 + math.exp(-float(np.float32(x))))


AMAX = float(np.float32(0.99))      # rendering constants reach both implementations as float32
AMIN = float(np.float32(1 / 255))


CAM = Camera(128.0, 128.0, 64.0, 48.0, 128, 96)   # f = 128 so pixel centres are dyadic ray slopes
NOEPS = O.Params(eps2d=0.0)


def on_pixel(u, v, tz, cam=CAM):
    """World point (camera at origin, R = I) that projects exactly onto pixel centre (u+.5, v+.5)."""
    return [(u + 0.5 - cam.cx) / cam.fx * tz, (v + 0.5 - cam.cy) / cam.fy * tz, tz]


# ----------------------------------------------------------------------------- exp / log
def test_ex32_lg32_against_libm():
    xs = np.linspace(-80, 80, 20001, dtype=np.float32)
    ex = np.array([O.ex32(x) for x in xs[::7]], np.float64)
    ref = np.exp(xs[::7].astype(np.float64))
    assert np.max(np.abs(ex / ref - 1)) < 3e-7          # ~2.5 ulp of float32
    ys = np.exp(np.linspace(-20, 20, 4001)).astype(np.float32)
    lg = np.array([O.lg32(y) for y in ys], np.float64)
    ref = np.log(ys.astype(np.float64))
    err = np.abs(lg - ref) / np.maximum(np.abs(ref), 1.0)
    assert err.max() < 3e-7


# ----------------------------------------------------------------------------- lone Gaussian
@pytest.mark.parametrize("logit", [0.3, 6.0])      # below and above the 0.99 opacity clamp
def test_lone_gaussian_at_its_centre(logit):
    u0, v0, tz = 40, 30, 2.0
    g = gmap_from([on_pixel(u0, v0, tz)], [[-2.5, -2.0, -2.2]], [[0.9, 0.1, -0.3, 0.2]], [logit],
                  [[0.2, 0.5, 0.9]], [0.7])
    r = O.render(g, [CAM], O.Params(), pixels=[[0, u0, v0]])
    a = min(AMAX, sig(logit))
    np.testing.assert_allclose(r["rgb"][0], a * np.float32([0.2, 0.5, 0.9]).astype(float), rtol=1e-12)
    np.testing.assert_allclose(r["depth"][0], a * tz, rtol=1e-12)
    np.testing.assert_allclose(r["unc"][0], a * float(np.float32(0.7)), rtol=1e-12)
    np.testing.assert_allclose(r["T"][0], 1 - a, rtol=1e-12)
    assert r["last_id"][0] == 0 and r["n_contrib"][0] == 1


def test_off_centre_axis_aligned_falloff():
    """Axis-aligned Gaussian on the optical axis: Sigma_2D = (f/d)^2 diag(sx^2, sy^2) + eps I."""
    ls = np.float32([-2.0, -2.6, -1.9])
    tz, logit = 3.0, 0.4
    g = gmap_from([[0.0, 0.0, tz]], [ls], [[1, 0, 0, 0]], [logit], [[1, 1, 1]], [1.0])
    p = O.Params()
    eps = float(np.float32(p.eps2d))
    s = np.exp(ls.astype(np.float64))
    sxx = (CAM.fx / tz) ** 2 * s[0] ** 2 + eps
    syy = (CAM.fy / tz) ** 2 * s[1] ** 2 + eps
    pix = np.array([[0, 64 + du, 48 + dv] for du in (-9, -3, 0, 2, 7) for dv in (-5, 0, 4)], np.int32)
    r = O.render(g, [CAM], p, pixels=pix)
    dx = pix[:, 1] + 0.5 - 64.0
    dy = pix[:, 2] + 0.5 - 48.0
    a = sig(logit) * np.exp(-0.5 * (dx ** 2 / sxx + dy ** 2 / syy))
    a = np.where(a < AMIN, 0.0, np.minimum(a, AMAX))
    np.testing.assert_allclose(r["unc"], a, rtol=1e-12, atol=1e-15)


def test_ewa_off_axis_closed_form():
    """Off-axis axis-aligned Gaussian: J has the -f t_x / t_z^2 term (2D covariance in closed form)."""
    ls = np.float32([-2.2, -2.4, -1.6])
    tx, tz = 0.75, 2.5
    g = gmap_from([[tx, 0.0, tz]], [ls], [[1, 0, 0, 0]], [1.0], [[1, 1, 1]], [1.0])
    pr = O.project(g, [CAM], NOEPS)
    s2 = np.exp(2 * ls.astype(np.float64))
    f = CAM.fx
    sxx = (f / tz) ** 2 * s2[0] + (f * tx / tz ** 2) ** 2 * s2[2]
    syy = (f / tz) ** 2 * s2[1]
    np.testing.assert_allclose(pr["cov2d"][0, 0], [sxx, 0.0, syy], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pr["mean2d"][0, 0], [f * tx / tz + CAM.cx, CAM.cy], rtol=1e-14)


def test_paper_isotropic_formula_on_axis():
    """Sec. III: f_i(p) = alpha exp(-|p - mu_2D|^2 / (2 r_2D^2)), r_2D = f r / d (isotropic, on axis, no dilation)."""
    r_world, tz, logit = 0.04, 2.0, -0.2
    lr = float(np.float32(math.log(r_world)))
    g = gmap_from([[0.0, 0.0, tz]], [[lr, lr, lr]], [[0.3, 0.5, -0.1, 0.8]], [logit], [[1, 1, 1]], [1.0])
    pix = np.array([[0, 64 + du, 48 + dv] for du in range(-6, 6) for dv in range(-6, 6)], np.int32)
    r = O.render(g, [CAM], NOEPS, pixels=pix)
    r2d = CAM.fx * math.exp(lr) / tz
    d2 = (pix[:, 1] + 0.5 - 64.0) ** 2 + (pix[:, 2] + 0.5 - 48.0) ** 2
    f = sig(logit) * np.exp(-d2 / (2 * r2d ** 2))
    f = np.where(f < AMIN, 0.0, f)
    np.testing.assert_allclose(r["unc"], f, rtol=1e-11, atol=1e-15)


# ----------------------------------------------------------------------------- several Gaussians
def test_three_gaussians_hand_expanded_front_to_back():
    u0, v0 = 70, 50
    depths = [3.0, 2.0, 4.0]                       # ids are not in depth order
    logits = [0.5, -0.3, 1.2]
    cols = [[0.9, 0.1, 0.2], [0.3, 0.8, 0.4], [0.1, 0.2, 0.95]]
    us = [0.25, 0.5, 0.75]
    g = gmap_from([on_pixel(u0, v0, d) for d in depths], [[-2.3, -2.3, -2.3]] * 3, [[1, 0, 0, 0]] * 3,
                  logits, cols, us)
    r = O.render(g, [CAM], O.Params(), pixels=[[0, u0, v0]])
    a = [sig(l) for l in logits]
    c = np.float32(cols).astype(float)
    order = [1, 0, 2]                              # by depth
    T, rgb, dep, unc = 1.0, np.zeros(3), 0.0, 0.0
    for i in order:
        rgb += a[i] * T * c[i]
        dep += a[i] * T * depths[i]
        unc += a[i] * T * float(np.float32(us[i]))
        T *= 1 - a[i]
    np.testing.assert_allclose(r["rgb"][0], rgb, rtol=1e-12)
    np.testing.assert_allclose(r["depth"][0], dep, rtol=1e-12)
    np.testing.assert_allclose(r["unc"][0], unc, rtol=1e-12)
    np.testing.assert_allclose(r["T"][0], T, rtol=1e-12)
    assert r["last_id"][0] == 2 and r["n_contrib"][0] == 3


def test_equal_depth_ties_break_by_id():
    u0, v0 = 20, 20
    g = gmap_from([on_pixel(u0, v0, 2.0)] * 2, [[-2.3] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.0, 0.0],
                  [[1, 0, 0], [0, 1, 0]], [0, 0])
    r = O.render(g, [CAM], O.Params(), pixels=[[0, u0, v0]])
    np.testing.assert_allclose(r["rgb"][0], [0.5, 0.25, 0.0], rtol=1e-12)   # id 0 in front


def test_termination_before_sixth_layer():
    """alpha = 0.8 layers: T after 5 = 0.2^5 = 3.2e-4 >= 1e-4 > 0.2^6, so layer 6 is never added."""
    u0, v0 = 60, 40
    n = 8
    logit = float(np.float32(math.log(4.0)))       # sigmoid = 0.8
    cols = np.random.default_rng(0).uniform(size=(n, 3))
    g = gmap_from([on_pixel(u0, v0, 1.0 + 0.5 * k) for k in range(n)], [[-2.0] * 3] * n, [[1, 0, 0, 0]] * n,
                  [logit] * n, cols, [1.0] * n)
    r = O.render(g, [CAM], O.Params(), pixels=[[0, u0, v0]])
    a = sig(logit)
    assert r["n_contrib"][0] == 5 and r["last_id"][0] == 4
    np.testing.assert_allclose(r["T"][0], (1 - a) ** 5, rtol=1e-12)
    c = np.float32(cols).astype(float)
    exp_rgb = sum(a * (1 - a) ** k * c[k] for k in range(5))
    np.testing.assert_allclose(r["rgb"][0], exp_rgb, rtol=1e-12)


def test_weights_plus_transmittance_is_one():
    """Constant colour k gives k (1 - T); all Gaussians at depth z give z (1 - T)."""
    cam = Camera(40.0, 40.0, 24.0, 16.0, 48, 32)
    g = random_scene(5, 300, [cam])
    g.rgb[:, :3] = 0.625
    g.su[:, 3] = 1.0
    g.mo[:, 2] = 2.75
    im = O.render_images(g, [cam])[0]
    assert (im["n_contrib"] > 0).mean() > 0.5
    np.testing.assert_allclose(im["rgb"], np.repeat(0.625 * (1 - im["T"])[..., None], 3, axis=2), atol=1e-12)
    np.testing.assert_allclose(im["unc"], 1 - im["T"], atol=1e-12)
    np.testing.assert_allclose(im["depth"], 2.75 * (1 - im["T"]), atol=1e-11)
    ig, _ = O.info_gain(g, [cam])
    np.testing.assert_allclose(ig[0], np.mean(1 - im["T"]), rtol=1e-12)


# ----------------------------------------------------------------------------- projection vs libraries
def test_projection_against_scipy_rotation_and_numeric_jacobian():
    rng = np.random.default_rng(3)
    cam_R = Rotation.from_euler("xyz", [0.2, -0.4, 0.3]).as_matrix()
    cam_T = np.array([0.3, -0.2, -1.0])
    cam = Camera(300.0, 280.0, 160.0, 120.0, 320, 240, cam_R, cam_T)
    n = 64
    t_cam = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.6, 0.6, n), rng.uniform(2, 6, n)], 1)
    mu = (cam.R.astype(float) @ t_cam.T).T + cam.T.astype(float)
    q = rng.normal(size=(n, 4))
    ls = rng.normal(-3, 0.5, size=(n, 3))
    g = gmap_from(mu, ls, q, rng.normal(size=n) + 1.0, rng.uniform(size=(n, 3)), rng.uniform(size=n))
    p = O.Params()
    pr = O.project(g, [cam], p)
    assert pr["vis"].all()
    R = cam.R.astype(float)
    T = cam.T.astype(float)
    K = np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1.0]])
    eps = float(np.float32(p.eps2d))
    for i in range(n):
        m = g.mo[i, :3].astype(float)
        t = R.T @ (m - T)
        uvw = K @ t
        np.testing.assert_allclose(pr["mean2d"][0, i], uvw[:2] / uvw[2], rtol=1e-12)
        np.testing.assert_allclose(pr["depth"][0, i], t[2], rtol=1e-12)
        qq = g.q[i].astype(float)
        Rq = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()   # scipy is scalar-last
        S3 = Rq @ np.diag(np.exp(2 * g.su[i, :3].astype(float))) @ Rq.T
        proj = lambda tt: np.array([cam.fx * tt[0] / tt[2] + cam.cx, cam.fy * tt[1] / tt[2] + cam.cy])
        h = 1e-6
        J = np.stack([(proj(t + h * e) - proj(t - h * e)) / (2 * h) for e in np.eye(3)], 1)
        C2 = J @ R.T @ S3 @ R @ J.T + eps * np.eye(2)
        np.testing.assert_allclose(pr["cov2d"][0, i], [C2[0, 0], C2[0, 1], C2[1, 1]], rtol=1e-7,
                                   atol=1e-7 * abs(C2).max())
        conic = pr["conic"][0, i]
        Cm = np.array([[conic[0], conic[1]], [conic[1], conic[2]]])
        Sm = np.array([[pr["cov2d"][0, i, 0], pr["cov2d"][0, i, 1]], [pr["cov2d"][0, i, 1], pr["cov2d"][0, i, 2]]])
        np.testing.assert_allclose(Cm @ Sm, np.eye(2), atol=1e-12)


def test_support_rect_covers_every_pixel_above_alpha_min():
    """The FP32 tile rectangle contains every pixel whose FP64 alpha clears the skip threshold."""
    cam = Camera(60.0, 60.0, 40.0, 30.0, 80, 60)
    g = random_scene(11, 400, [cam], box=((-2, -1.5, 0.5), (2, 1.5, 4)), log_scale=(-2.5, 0.7))
    p = O.Params(tile_w=8, tile_h=8)
    pr = O.project(g, [cam], p)
    vv, uu = np.meshgrid(np.arange(cam.height) + 0.5, np.arange(cam.width) + 0.5, indexing="ij")
    amin = float(np.float32(p.alpha_min))
    checked = 0
    for i in np.nonzero(pr["vis"][0])[0]:
        mx, my = pr["mean2d"][0, i]
        a, b, c = pr["conic"][0, i]
        dx, dy = uu - mx, vv - my
        al = pr["opac"][0, i] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
        ys, xs = np.nonzero(al >= amin * (1 + 1e-5))
        x0, y0, x1, y1 = pr["rect"][0, i]
        if len(xs):
            checked += 1
            assert (xs // 8 >= x0).all() and (xs // 8 < x1).all() and (ys // 8 >= y0).all() and (ys // 8 < y1).all()
    assert checked > 100


def test_opacity_floor_and_near_plane():
    cam = Camera(60.0, 60.0, 40.5, 30.5, 80, 60)     # the Gaussians sit exactly on a pixel centre
    n = 200
    logit = np.linspace(-5.6, -5.47, n)             # straddles -ln 254
    g = gmap_from([[0, 0, 2.0]] * n, [[-2.0] * 3] * n, [[1, 0, 0, 0]] * n, logit, [[1, 1, 1]] * n, [1] * n)
    pr = O.project(g, [cam])
    o = 1 / (1 + np.exp(-g.mo[:, 3].astype(float)))
    far = np.abs(o * 255 - 1) > 1e-5
    np.testing.assert_array_equal(pr["vis"][0].astype(bool)[far], (o * 255 >= 1)[far])
    z = np.float32([0.1, 0.2, 0.2000001, 0.3])
    g2 = gmap_from([[0, 0, zz] for zz in z], [[-4.0] * 3] * 4, [[1, 0, 0, 0]] * 4, [3.0] * 4, [[1, 1, 1]] * 4, [1] * 4)
    np.testing.assert_array_equal(O.project(g2, [cam])["vis"][0], [0, 0, 1, 1])


# ----------------------------------------------------------------------------- guard band
# The cull of a centre outside the guard band (the reading taken where the paper is silent:
# 1.3 times the half field of view on each axis, |t_x / t_z| <= 1.3 (W/2) / f_x and the same
# in y).  fx != fy and W/fx != H/fy, so that a swap of the axes, of W and H or of fx and fy
# moves one of the bands; the factor 1.3 is written out here, not taken from Params.
GUARD_READING = 1.3
GUARD_CAM = Camera(120.0, 100.0, 64.0, 48.0, 128, 96)
GUARD_LS = -1.2          # sigma 0.30 m: the support reaches into the image from inside the band


def guard_band_scene(cam=GUARD_CAM, depths=(1.5, 2.5, 4.0), rel=1e-3):
    """One Gaussian per (depth, axis, side, factor): centre at t_axis / t_z = side x factor x the
    band's slope, the other lateral coordinate 0, factor 1 - rel (inside) or 1 + rel (outside).
    Returns the map and, per Gaussian, (axis, side, factor, t_z, inside)."""
    slope = (GUARD_READING * (cam.width / 2) / cam.fx, GUARD_READING * (cam.height / 2) / cam.fy)
    pos, meta = [], []
    for tz in depths:
        for axis in (0, 1):
            for side in (1.0, -1.0):
                for f in (1 - rel, 1 + rel):
                    t = [0.0, 0.0, tz]
                    t[axis] = side * f * slope[axis] * tz
                    pos.append(t)
                    meta.append((axis, side, f, tz, f < 1))
    n = len(pos)
    g = gmap_from(pos, [[GUARD_LS] * 3] * n, [[1, 0, 0, 0]] * n, [2.0] * n, [[0.25, 0.5, 0.75]] * n, [1.0] * n)
    return g, meta


def _axis_aligned_alpha(g, i, cam, pix, eps):
    """Closed-form alpha of Gaussian i (identity rotation, camera at the origin looking +z) at
    the pixel centres pix (K x 3: view, u, v): Sigma_2D = J diag(s^2) J^T + eps I with
    J = [[f_x/t_z, 0, -f_x t_x/t_z^2], [0, f_y/t_z, -f_y t_y/t_z^2]]; the skip and clamp rules."""
    tx, ty, tz = g.mo[i, :3].astype(np.float64)
    s2 = np.exp(2 * g.su[i, :3].astype(np.float64))
    fx, fy = cam.fx, cam.fy
    J = np.array([[fx / tz, 0, -fx * tx / tz ** 2], [0, fy / tz, -fy * ty / tz ** 2]])
    S = J @ np.diag(s2) @ J.T + eps * np.eye(2)
    mx, my = fx * tx / tz + cam.cx, fy * ty / tz + cam.cy
    d = np.stack([pix[:, 1] + 0.5 - mx, pix[:, 2] + 0.5 - my], 1)
    q = np.einsum("ki,ij,kj->k", d, np.linalg.inv(S), d)
    a = sig(g.mo[i, 3]) * np.exp(-0.5 * q)
    return np.where(a < AMIN, 0.0, np.minimum(a, AMAX))


def test_guard_band_keeps_inside_culls_outside():
    g, meta = guard_band_scene()
    pr = O.project(g, [GUARD_CAM])
    np.testing.assert_array_equal(pr["vis"][0].astype(bool), [m[4] for m in meta])


def test_guard_band_edge_gaussian_closed_form_alpha():
    """A centre outside the image but inside the band is rendered, with the closed-form alpha
    of its 2D Gaussian at every pixel; a centre just outside the band adds nothing anywhere."""
    g, meta = guard_band_scene()
    p = O.Params()
    eps = float(np.float32(p.eps2d))
    pix = O.all_pixels([GUARD_CAM])
    for i, (axis, side, f, tz, inside) in enumerate(meta):
        one = g.subset([i])
        r = O.render(one, [GUARD_CAM], p, pixels=pix)
        if inside:
            mx = GUARD_CAM.fx * float(one.mo[0, 0]) / float(one.mo[0, 2]) + GUARD_CAM.cx
            my = GUARD_CAM.fy * float(one.mo[0, 1]) / float(one.mo[0, 2]) + GUARD_CAM.cy
            assert not (0 <= mx <= GUARD_CAM.width and 0 <= my <= GUARD_CAM.height), "centre must be off-image"
            a = _axis_aligned_alpha(g, i, GUARD_CAM, pix, eps)
            assert (a > 0).sum() > 20, "the support must reach into the image"
            np.testing.assert_allclose(r["unc"], a, rtol=1e-11, atol=1e-15)
            np.testing.assert_allclose(r["T"], 1 - a, rtol=1e-11, atol=1e-15)
        else:
            assert (r["unc"] == 0).all() and (r["T"] == 1).all() and (r["n_contrib"] == 0).all()


# ----------------------------------------------------------------------------- binning / sort
def test_bin_sort_against_brute_force():
    from paper_2409_18122_gb300.scenes import synthetic_records
    cams = [Camera(50, 50, 20, 20, 40, 40), Camera(50, 50, 40, 30, 80, 56), Camera(50, 50, 8, 8, 16, 16)]
    rec = synthetic_records(4, 60, cams, tile_w=16, tile_h=16, max_extent=4, tie_frac=0.3)
    rec["dkey"] = rec["depth"].view(np.uint32)
    b = O.bin_sort(rec, cams)
    tx, base = O.tile_grid(cams)
    pairs = []
    for r in range(len(rec["gid"])):
        v = int(rec["view"][r])
        x0, y0, x1, y1 = rec["rect"][r]
        for y in range(y0, y1):
            for x in range(x0, x1):
                gt = int(base[v]) + y * int(tx[v]) + x
                pairs.append((gt, float(rec["depth"][r]), r))
    pairs.sort()
    assert b["n_pairs"] == len(pairs)
    np.testing.assert_array_equal(b["vals"], [p[2] for p in pairs])
    np.testing.assert_array_equal(b["keys"] >> np.uint64(32), [p[0] for p in pairs])
    np.testing.assert_array_equal((b["keys"] & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32),
                                  np.float32([p[1] for p in pairs]))
    for t in range(int(base[-1])):
        idx = [i for i, p in enumerate(pairs) if p[0] == t]
        if idx:
            assert tuple(b["ranges"][t]) == (idx[0], idx[-1] + 1)
        else:
            assert tuple(b["ranges"][t]) == (0, 0)


def test_depth_key_bits_are_monotone():
    d = np.sort(np.random.default_rng(1).uniform(0.2, 100.0, 10000).astype(np.float32))
    k = d.view(np.uint32)
    assert (np.diff(k.astype(np.int64)) >= 0).all()


# ----------------------------------------------------------------------------- gradients
def _loss(g, cams, dimg, params, values):
    imgs = O.render_images(g, cams, params, values=values)
    L = 0.0
    for im, d in zip(imgs, dimg):
        L += np.sum(im["rgb"] * d[..., :3]) + np.sum(im["depth"] * d[..., 3])
    return L, [(im["n_contrib"].copy(), im["n_clamp"].copy()) for im in imgs]


def _fd_check(g, cams, params, seed, rtol, n_param_max=None):
    rng = np.random.default_rng(seed)
    dimg = [rng.normal(size=(c.height, c.width, 4)) for c in cams]
    an = O.grad(g, cams, dimg, params)
    base = [a.astype(np.float64) for a in (g.mo, g.su, g.q, g.rgb)]
    names = [("dmo", 0, range(4)), ("dsu", 1, range(3)), ("dq", 2, range(4)), ("drgb", 3, range(3))]
    checked = skipped = 0
    worst = 0.0
    scale = {k: max(np.abs(an[k]).max(), 1e-30) for k, _, _ in names}
    for key, ai, comps in names:
        for i in range(g.n):
            for c in comps:
                th = base[ai][i, c]
                h = 1e-6 * max(1.0, abs(th))
                vals_p = [b.copy() for b in base]
                vals_m = [b.copy() for b in base]
                vals_p[ai][i, c] += h
                vals_m[ai][i, c] -= h
                Lp, ep = _loss(g, cams, dimg, params, vals_p)
                Lm, em = _loss(g, cams, dimg, params, vals_m)
                if any((a[0] != b[0]).any() or (a[1] != b[1]).any() for a, b in zip(ep, em)):
                    skipped += 1
                    continue
                fd = (Lp - Lm) / (2 * h)
                a = an[key][i, c]
                err = abs(fd - a) / max(abs(a), 1e-3 * scale[key])
                worst = max(worst, err)
                assert err < rtol, (key, i, c, fd, a)
                checked += 1
    return checked, skipped, worst


def test_gradient_matches_finite_differences_standard_rules():
    cams = [Camera(30.0, 30.0, 16.0, 12.0, 32, 24),
            Camera(30.0, 30.0, 16.0, 12.0, 32, 24, Rotation.from_euler("y", 0.3).as_matrix(), [-0.5, 0.1, 0.2])]
    g = random_scene(21, 14, cams, box=((-1, -0.8, 2), (1, 0.8, 4)), log_scale=(-2.0, 0.3))
    checked, skipped, worst = _fd_check(g, cams, O.Params(), 7, 1e-5)
    assert checked > 0.8 * (checked + skipped) and checked > 100


def test_gradient_matches_finite_differences_smooth_rules():
    cams = [Camera(30.0, 30.0, 16.0, 12.0, 32, 24)]
    g = random_scene(22, 10, cams, box=((-1, -0.8, 2), (1, 0.8, 4)), log_scale=(-2.0, 0.3))
    checked, skipped, worst = _fd_check(g, cams, O.smooth_params(), 8, 1e-5)
    assert skipped == 0 and checked == 14 * 10


def test_gradient_colour_is_blend_weight():
    """dC/dc_i = w_i = alpha_i T_i: two Gaussians on one pixel centre."""
    u0, v0 = 30, 20
    logits = [0.2, -0.4]
    g = gmap_from([on_pixel(u0, v0, 2.0), on_pixel(u0, v0, 3.0)], [[-2.2] * 3] * 2, [[1, 0, 0, 0]] * 2, logits,
                  [[0.3, 0.3, 0.3]] * 2, [0, 0])
    d = np.zeros((CAM.height, CAM.width, 4))
    d[v0, u0, 0] = 1.0
    gr = O.grad(g, [CAM], [d])
    a0, a1 = sig(logits[0]), sig(logits[1])
    np.testing.assert_allclose(gr["drgb"][:, 0], [a0, (1 - a0) * a1], rtol=1e-12)
    np.testing.assert_allclose(gr["drgb"][:, 1:], 0)


def test_gradient_opacity_single_gaussian():
    """Below the clamp: dC/do = exp(-q/2) c, so dC/dlogit = exp(-q/2) c o (1 - o)."""
    logit, col = 0.1, 0.6
    g = gmap_from([[0.0, 0.0, 2.5]], [[-2.0, -2.3, -2.1]], [[0.8, 0.2, 0.1, -0.3]], [logit], [[col, 0, 0]], [0])
    pix = (70, 45)
    d = np.zeros((CAM.height, CAM.width, 4))
    d[pix[1], pix[0], 0] = 1.0
    pr = O.project(g, [CAM])
    mx, my = pr["mean2d"][0, 0]
    a, b, c = pr["conic"][0, 0]
    dx, dy = pix[0] + 0.5 - mx, pix[1] + 0.5 - my
    G = math.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
    o = sig(logit)
    assert o * G > 1 / 255
    gr = O.grad(g, [CAM], [d])
    np.testing.assert_allclose(gr["dmo"][0, 3], G * float(np.float32(col)) * o * (1 - o), rtol=1e-12)


# ------------------------------------------------------------ render-free view utility (Sec. IV-A/B)
def _mo(xyz):
    a = np.zeros((len(xyz), 4), np.float32)
    a[:, :3] = np.asarray(xyz, np.float32)
    return a


def test_uncertainty_update_closed_form_and_bookkeeping():
    prev = _mo([[0, 0, 0], [1, 1, 1], [2, 0, 0]])
    cur = _mo([[3, 4, 0], [1, 1, 1], [2, 0, 0.5]])
    u0 = np.array([7.0, 7.0, 7.0])
    np.testing.assert_allclose(O.uncertainty_update(prev, cur, u0), [5.0, 7.0, 0.5])
    np.testing.assert_allclose(O.uncertainty_update(prev, cur, u0, squared=True), [25.0, 7.0, 0.25])


def test_uncertainty_thresholds_hand_values():
    """u = 0, 1, ..., 9: mean 4.5, population variance 8.25; G_H = {6..9}, G_L = {0..3}."""
    u = np.arange(10.0)
    mo = _mo([[0, 0, 1]] * 10)
    mean, sigma, t_hi, t_lo, m = O.uncertainty_thresholds(mo, u)
    assert (mean, m) == (4.5, 10)
    assert sigma == pytest.approx(math.sqrt(8.25), rel=1e-15)
    assert sum(u > t_hi) == 4 and sum(u < t_lo) == 4 and u[u > t_hi].min() == 6 and u[u < t_lo].max() == 3
    # ground-plane removal: the five lowest Gaussians are left out
    mo2 = mo.copy()
    mo2[:5, 2] = -1.0
    mean2, sigma2, _, _, m2 = O.uncertainty_thresholds(mo2, u, ground_z=0.0)
    assert (mean2, m2) == (7.0, 5) and sigma2 == pytest.approx(math.sqrt(2.0), rel=1e-15)


def test_visibility_pinhole_edges_and_range():
    cam = Camera(100.0, 100.0, 50.0, 40.0, 100, 80)           # camera at the origin looking along +z
    # u = 100 x / z + 50: x = -1.5 at z = 3 gives u = 0 (inside), x = 1.5 gives u = 100 (outside);
    # v = 100 y / z + 40 with y = -+1.25, z = 3.125 gives exactly 0 (inside) and 80 (outside)
    pts = [[0, 0, 3], [0, 0, 6], [0, 0, -1], [-1.5, 0, 3], [1.5, 0, 3], [1.4999, 0, 3], [0, 1.25, 3.125],
           [0, -1.25, 3.125], [0, 0, 5.0], [0, 0, 0.2]]
    vis = O.visibility(_mo(pts), cam, near_plane=0.2, range_m=5.0)
    np.testing.assert_array_equal(vis, [1, 0, 0, 1, 0, 1, 0, 1, 1, 0])


def test_visibility_fp32_decisions_match_fp64_projection_away_from_edges():
    """The float32 decision sequence against an independent FP64 pinhole projection, on
    random points that are not within 1e-3 of an image edge or a depth limit."""
    rng = np.random.default_rng(3)
    cam = Camera(200.0, 210.0, 80.0, 60.0, 160, 120, Rotation.from_euler("xyz", [0.2, -0.5, 0.3]).as_matrix(),
                 [0.3, -0.2, 0.5])
    R = np.asarray(cam.R, np.float64)
    # points around the frustum: camera coordinates with |t_x|, |t_y| up to 0.7 t_z, t_z in (0.1, 6)
    tz = rng.uniform(0.1, 6.0, 20000)
    tc = np.stack([rng.uniform(-0.7, 0.7, 20000) * tz, rng.uniform(-0.7, 0.7, 20000) * tz, tz], 1)
    p = tc @ R.T + np.asarray(cam.T, np.float64)
    t = (p - np.asarray(cam.T, np.float64)) @ R          # t = R^T (p - T)
    px = cam.fx * t[:, 0] / t[:, 2] + cam.cx
    py = cam.fy * t[:, 1] / t[:, 2] + cam.cy
    ref = (t[:, 2] > 0.2) & (t[:, 2] <= 5.0) & (px >= 0) & (px < cam.width) & (py >= 0) & (py < cam.height)
    clear = (np.abs(t[:, 2] - 0.2) > 1e-3) & (np.abs(t[:, 2] - 5.0) > 1e-3) & (np.abs(px) > 1e-3) & \
            (np.abs(px - cam.width) > 1e-3) & (np.abs(py) > 1e-3) & (np.abs(py - cam.height) > 1e-3)
    got = O.visibility(_mo(p), cam, 0.2, 5.0)
    assert ref[clear].sum() > 2000 and (~ref[clear]).sum() > 2000
    np.testing.assert_array_equal(got[clear], ref[clear])


def test_view_utility_hand_counts():
    """Ten visible Gaussians with u = 0..9 and five more behind the camera: xi = 4 - lambda * 4
    (G_H = {6..9}, G_L = {0..3}, thresholds from all fifteen), and the sum mode adds u of the
    visible ones."""
    cam = Camera(100.0, 100.0, 50.0, 40.0, 100, 80)
    vis_pts = [[0.1 * i - 0.5, 0, 3] for i in range(10)]
    hid_pts = [[0, 0, -2]] * 5
    mo = _mo(vis_pts + hid_pts)
    u = np.concatenate([np.arange(10.0), np.array([0.0, 9.0, 4.5, 4.5, 4.5])])
    st = O.uncertainty_thresholds(mo, u)
    assert sum(u > st[2]) == 5 and sum(u < st[3]) == 5       # the hidden 9 and 0 join G_H and G_L
    xi, counts = O.view_utility(mo, u, [cam], lam=1.0)
    np.testing.assert_array_equal(counts, [[4, 4]])
    assert xi[0] == 0.0
    xi2, _ = O.view_utility(mo, u, [cam], lam=0.5)
    assert xi2[0] == 2.0
    xs, _ = O.view_utility(mo, u, [cam], mode="sum")
    assert xs[0] == 45.0


def test_region_uncertainty_hand_means():
    mo = _mo([[0.5, 0.5, 0.5], [1.0, 2.0, 0.1], [3.0, 0.1, 0.1], [2.6, 2.6, 0.2], [-0.1, 0, 0], [9, 9, 9]])
    u = np.array([1.0, 3.0, 5.0, 7.0, 100.0, 100.0])
    mean, cnt = O.region_uncertainty(mo, u, origin=(0, 0, 0), size=2.5, dims=(2, 2, 1))
    # region (0,0): first two; (1,0): the third; (1,1): the fourth; the last two lie outside
    np.testing.assert_array_equal(cnt, [2, 1, 0, 1])
    np.testing.assert_allclose(mean, [2.0, 5.0, 0.0, 7.0])


def test_trajectory_utility_hand_sums_and_first_argmax():
    """Three trajectories of two states; state utilities known by construction: a pose that
    sees the two highest-u Gaussians, one that sees the two lowest, one that sees nothing."""
    mo = _mo([[0, 0, 3], [0.1, 0, 3], [0, 0, -3], [0.1, 0, -3], [5, 5, 5], [5, 5, 6]])
    u = np.array([9.0, 8.0, 0.0, 1.0, 4.0, 5.0])      # mean 4.5, sigma ~3.3: G_H = {9, 8}, G_L = {0, 1}
    see_hi = Camera(100.0, 100.0, 50.0, 40.0, 100, 80)
    see_lo = Camera(100.0, 100.0, 50.0, 40.0, 100, 80, Rotation.from_euler("y", np.pi).as_matrix(), [0, 0, 0])
    blind = Camera(100.0, 100.0, 50.0, 40.0, 100, 80, np.eye(3), [0, 0, 50])
    cams = [see_hi, blind, see_lo, see_lo, see_hi, see_lo]      # xi: 2, 0 | -2, -2 | 2, -2
    s, best = O.trajectory_utility(mo, u, cams, 3, 2)
    np.testing.assert_array_equal(s, [2.0, -4.0, 0.0])
    assert best == 0
    s2, best2 = O.trajectory_utility(mo, u, [see_hi, see_hi, blind, blind, see_hi, see_hi], 3, 2)
    assert list(s2) == [4.0, 0.0, 4.0] and best2 == 0             # ties: the first


def test_collision_check_closed_form():
    """One Gaussian at the origin with principal axis 0.2 m: gamma = 0.3 + 3 * 0.2 = 0.9 m."""
    mo = _mo([[0, 0, 0], [10, 0, 0]])
    su = np.zeros((2, 4), np.float32)
    su[0, :3] = np.log([0.1, 0.2, 0.05])
    su[1, :3] = np.log([0.01, 0.01, 0.01])
    pts = np.zeros((4, 4), np.float32)
    pts[:, 0] = [0.5, 1.0, 9.95, 5.0]
    margin, hit = O.collision_check(mo, su, pts, r_robot=0.3, lambda_g=3.0)
    r0 = float(O.ex32(np.log(np.float32(0.2))))
    g0, g1 = 0.3 + 3 * r0, 0.3 + 3 * float(O.ex32(np.log(np.float32(0.01))))
    np.testing.assert_allclose(margin, [0.5 - g0, 1.0 - g0, 0.05 - g1, min(5.0 - g0, 5.0 - g1)], rtol=1e-6)
    np.testing.assert_array_equal(hit, [True, False, True, False])
    m2, h2 = O.collision_check(mo, su, pts, 0.3, 3.0, ground_z=5.0)     # every Gaussian removed
    assert np.isinf(m2).all() and not h2.any()


# ------------------------------------------------------------------ mapping loss (Eq. 3)
def _ssim_brute(x, y, r=5, sigma=1.5):
    """SSIM map by explicit window sums (zero outside the image), straight from the definition."""
    H, W = x.shape
    w = {(i, j): math.exp(-(i * i + j * j) / (2 * sigma * sigma)) for i in range(-r, r + 1) for j in range(-r, r + 1)}
    tot = sum(w.values())
    out = np.zeros_like(x)
    for py in range(H):
        for px in range(W):
            m = [0.0] * 5
            for (i, j), wt in w.items():
                yy, xx = py + i, px + j
                if 0 <= yy < H and 0 <= xx < W:
                    a, b = x[yy, xx], y[yy, xx]
                    for k, v in enumerate((a, b, a * a, b * b, a * b)):
                        m[k] += wt / tot * v
            mx, my = m[0], m[1]
            sx, sy, sxy = m[2] - mx * mx, m[3] - my * my, m[4] - mx * my
            c1, c2 = 0.01 ** 2, 0.03 ** 2
            out[py, px] = (2 * mx * my + c1) * (2 * sxy + c2) / ((mx * mx + my * my + c1) * (sx + sy + c2))
    return out


def test_ssim_map_brute_force_tiny():
    rng = np.random.default_rng(31)
    x, y = rng.uniform(0, 1, (7, 9)), rng.uniform(0, 1, (7, 9))
    np.testing.assert_allclose(O.ssim_map(x, y), _ssim_brute(x, y), rtol=1e-12, atol=1e-14)


def test_ssim_moments_match_scipy_gaussian_filter():
    """The windowed moments equal scipy's Gaussian filter truncated at radius 5, zero outside."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(32)
    x, y = rng.uniform(0, 1, (20, 27)), rng.uniform(0, 1, (20, 27))
    f = lambda a: gaussian_filter(a, 1.5, mode="constant", cval=0.0, truncate=5 / 1.5)
    mx, my = f(x), f(y)
    ref = ((2 * mx * my + 1e-4) * (2 * (f(x * y) - mx * my) + 9e-4)) / \
        ((mx * mx + my * my + 1e-4) * (f(x * x) - mx * mx + f(y * y) - my * my + 9e-4))
    np.testing.assert_allclose(O.ssim_map(x, y), ref, rtol=1e-12, atol=1e-14)


def test_ssim_constant_images_interior_closed_form():
    """Constant images a, b: away from the border sigma = 0 and S = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.7, 0.3
    s = O.ssim_map(np.full((16, 16), a), np.full((16, 16), b))
    np.testing.assert_allclose(s[5:-5, 5:-5], (2 * a * b + 1e-4) / (a * a + b * b + 1e-4), rtol=1e-13)


def test_mapping_loss_identical_images():
    """x = y: L1 terms vanish, SSIM = 1 exactly (loss 0) and, SSIM being maximal there, its gradient is 0."""
    rng = np.random.default_rng(33)
    x = rng.uniform(0, 1, (3, 12, 15))
    d = rng.uniform(1, 3, (12, 15))
    L, gr, gd = O.mapping_loss(x, d, x, d)
    assert abs(L) < 1e-14
    assert np.abs(gr).max() < 1e-12 and np.abs(gd).max() == 0.0


def test_mapping_loss_l1_weights_reduce_to_plain_means():
    """w = (0.1, 1/3, 0) is mean |rgb - ref| over all elements + 0.1 mean |d - ref|."""
    rng = np.random.default_rng(34)
    x, y = rng.uniform(0, 1, (3, 10, 11)), rng.uniform(0, 1, (3, 10, 11))
    d, dr = rng.uniform(1, 3, (10, 11)), rng.uniform(1, 3, (10, 11))
    L, gr, gd = O.mapping_loss(x, d, y, dr, w_d=0.1, w_c=1 / 3, w_s=0.0)
    assert L == pytest.approx(np.abs(x - y).mean() + 0.1 * np.abs(d - dr).mean(), rel=1e-14)
    np.testing.assert_allclose(gr, np.sign(x - y) / x.size, rtol=1e-14)
    np.testing.assert_allclose(gd, 0.1 * np.sign(d - dr) / d.size, rtol=1e-14)


def test_mapping_loss_gradient_central_differences():
    """dL/d(rgb, depth) of Eq. 3 against FP64 central differences (the L1 kinks are avoided: |x - y| >= 0.02)."""
    rng = np.random.default_rng(35)
    y = rng.uniform(0.1, 0.9, (3, 9, 13))
    x = y + rng.choice([-1, 1], y.shape) * rng.uniform(0.02, 0.2, y.shape)
    dr = rng.uniform(1, 3, (9, 13))
    d = dr + rng.choice([-1, 1], dr.shape) * rng.uniform(0.02, 0.2, dr.shape)
    L, gr, gd = O.mapping_loss(x, d, y, dr)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 4, 6), (2, 8, 12), (0, 3, 11), (2, 0, 7)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (O.mapping_loss(xp, d, y, dr)[0] - O.mapping_loss(xm, d, y, dr)[0]) / (2 * h)
        assert gr[idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    for idx in [(0, 0), (5, 7)]:
        dp, dm = d.copy(), d.copy()
        dp[idx] += h
        dm[idx] -= h
        fd = (O.mapping_loss(x, dp, y, dr)[0] - O.mapping_loss(x, dm, y, dr)[0]) / (2 * h)
        assert gd[idx] == pytest.approx(fd, rel=1e-6)


def test_mapping_loss_views_normalisation():
    """N_p over all views: one view reduces to mapping_loss; a view repeated twice has the same
    loss with half the gradient per copy; the three reported terms recombine to L."""
    rng = np.random.default_rng(36)
    x, y = rng.uniform(0, 1, (3, 8, 10)), rng.uniform(0, 1, (3, 8, 10))
    d, dr = rng.uniform(1, 3, (8, 10)), rng.uniform(1, 3, (8, 10))
    L1v, gr1, gd1 = O.mapping_loss(x, d, y, dr)
    L, l1d, l1c, ss, gr, gd = O.mapping_loss_views([x], [d], [y], [dr])
    assert L == pytest.approx(L1v, rel=1e-15) and np.array_equal(gr[0], gr1)
    L2, l1d2, l1c2, ss2, gr2, gd2 = O.mapping_loss_views([x, x], [d, d], [y, y], [dr, dr])
    assert L2 == pytest.approx(L1v, rel=1e-14) and ss2 == pytest.approx(ss, rel=1e-14)
    np.testing.assert_allclose(gr2[1], gr1 / 2, rtol=1e-15)
    assert L == pytest.approx(l1d + 0.4 * l1c + 0.1 * (1 - ss), rel=1e-14)


def test_adam_first_steps_by_hand():
    """Adam from zero moments: the first step moves each parameter by lr g / (|g| + eps), i.e.
    lr times the sign of g up to eps; the second step, with the bias corrections written out by
    hand, and a zero gradient that leaves the parameter and the moments unchanged."""
    p = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 0.0, 1e-3])
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    p1, m1, v1 = O.adam_step(p, g, np.zeros(4), np.zeros(4), 1, lr, b1, b2, eps)
    np.testing.assert_allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    assert p1[2] == p[2] and m1[2] == 0 and v1[2] == 0
    g2 = np.array([-0.1, 2.0, 0.0, 1e-3])
    p2, m2, v2 = O.adam_step(p1, g2, m1, v1, 2, lr, b1, b2, eps)
    mm = 0.9 * 0.1 * g + 0.1 * g2
    vv = 0.999 * 0.001 * g * g + 0.001 * g2 * g2
    ref = p1 - lr / (1 - 0.81) * mm / (np.sqrt(vv) / np.sqrt(1 - 0.999 ** 2) + eps)
    np.testing.assert_allclose(m2, mm, rtol=1e-14)
    np.testing.assert_allclose(v2, vv, rtol=1e-14)
    np.testing.assert_allclose(p2, ref, rtol=1e-13)


def test_adam_matches_torch_cpu_adam():
    """Five steps against PyTorch's own CPU Adam in FP64 (a library implementation)."""
    import torch
    rng = np.random.default_rng(41)
    p0 = rng.normal(size=(64, 4))
    grads = [rng.normal(size=(64, 4)) * s for s in (1.0, 0.1, 3.0, 0.0, 1e-3)]
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=2e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for t, g in enumerate(grads, start=1):
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = O.adam_step(p, g, m, v, t, 2e-3)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)
