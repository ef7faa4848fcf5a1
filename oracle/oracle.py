"""Python front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  Nothing here is used by, or uses, the
CUDA path; inputs arrive as plain arrays or duck-typed camera objects with
attributes fx, fy, cx, cy, width, height, R (3x3, camera-to-world) and T.

Functions and the passages they follow (RT-GuIDE, arXiv 2409.18122):
  project      Sec. III projection mu_2D = K R^T (mu - T) / d, d = e3^T R^T (mu - T),
               generalised to the EWA 2D covariance; FP32 cull/key/rect decisions.
  render       Sec. III compositing C(p) = sum_i c_i f_i prod_{j<i} (1 - f_j), depth
               with d_i in place of c_i, uncertainty u_i (Sec. IV-A) likewise.
  grad         Eq. (2): gradient of a linear functional of the rendered images
               with respect to every map parameter (chain rule, FP64).
  info_gain    Eq. (nbv) with the binary-sparsity Jacobian (Sec. IV-A): per-view
               mean of the composited uncertainty channel.
  bin_sort     Sec. III "sorted in increasing order of depth": pairs (tile, Gaussian)
               ordered by (view, tile, depth, record index).
  uncertainty_update   Sec. IV-A: u = |mu_k - mu_{k-1}| (or its square), unchanged
               means keep their u.
  uncertainty_thresholds  Sec. IV-C (implementation details): G_H / G_L thresholds at
               half a standard deviation above / below the mean of u.
  visibility / view_utility  Sec. IV-B, Eq. view_util: xi = |visible G_H| - lambda
               |visible G_L| (or the sum of u of the visible Gaussians); visible =
               in the field of view and within the perception range.
  region_uncertainty   Sec. IV-B high-level planner: mean u of cuboid regions.
  trajectory_utility   Eq. traj_utility: sum of xi over a trajectory's states, best one.
  collision_check      Sec. IV-B collision checking: distance of each test point to every
               Gaussian against r_robot + lambda_g r (principal axis as the radius).
  ssim_map / mapping_loss  Eq. 3: L1 depth + lambda_1 L1 colour + lambda_2 (1 - SSIM), SSIM with
               the 11 x 11 Gaussian window (sigma 1.5, zero outside the image; the paper
               does not state the window), and the gradient with respect to the images.
  adam_step    the optimiser of the mapping iterations (Adam, as in the paper's mapping
               module): one update with bias corrections.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so from oracle.c with gcc (FP contraction off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        lib.or_num_threads.restype = I
        lib.ex32.argtypes = [ctypes.c_float]
        lib.ex32.restype = ctypes.c_float
        lib.or_ex32v.argtypes = [I64, P, P]
        lib.or_ex32v.restype = None
        lib.lg32.argtypes = [ctypes.c_float]
        lib.lg32.restype = ctypes.c_float
        lib.or_project.argtypes = [I64, P, P, P, P, P, P, I, P, P, P, P, P, P, P, P, P, P, P]
        lib.or_project.restype = None
        lib.or_render.argtypes = [I64, P, P, P, P, P, P, P, I, P, P, P, I64, P, D, P, P, P, P, P, P]
        lib.or_render.restype = None
        lib.or_grad.argtypes = [I64, P, P, P, P, P, P, P, I, P, P, P, I64, P, P, P, P, P, P, P]
        lib.or_grad.restype = None
        lib.or_bin_count.argtypes = [I64, P]
        lib.or_bin_count.restype = I64
        lib.or_bin.argtypes = [I64, P, P, P, P, P, I64, P, P, P]
        lib.or_bin.restype = None
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Params:
    """Rendering constants the paper leaves unstated (readings, see module doc of oracle.c)."""
    tile_w: int = 16
    tile_h: int = 16
    eps2d: float = 0.3
    near: float = 0.2
    guard: float = 1.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4

    def block(self) -> np.ndarray:
        # values pass through float32 exactly as the GPU receives them
        f = lambda x: float(np.float32(x))
        return np.array([self.tile_w, self.tile_h, f(self.eps2d), f(self.near), f(self.guard),
                         f(self.alpha_min), f(self.alpha_max), f(self.T_min)], np.float64)


def smooth_params(**kw) -> Params:
    """No discrete events: no skip, no stop, no clamp (for finite differences)."""
    p = Params(alpha_min=0.0, alpha_max=1.0, T_min=0.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def view_tile(c, params: Params):
    """Tile size of a view: the camera's own (attributes tile_w, tile_h, if non-zero) else the params'."""
    tw, th = getattr(c, "tile_w", 0), getattr(c, "tile_h", 0)
    return (tw, th) if tw and th else (params.tile_w, params.tile_h)


def _cams(cams, params: Params):
    V = len(cams)
    cf = np.zeros((V, 16), np.float32)
    wh = np.zeros((V, 4), np.int32)
    for v, c in enumerate(cams):
        cf[v, 0:4] = [c.fx, c.fy, c.cx, c.cy]
        cf[v, 4:13] = np.asarray(c.R, np.float32).reshape(9)
        cf[v, 13:16] = np.asarray(c.T, np.float32).reshape(3)
        wh[v] = [c.width, c.height, *view_tile(c, params)]
    return cf, wh


def _map(gmap, values=None):
    """FP32 arrays (decisions) and FP64 arrays (values; defaults to the FP32 ones promoted)."""
    m32 = [np.ascontiguousarray(a, np.float32) for a in (gmap.mo, gmap.su, gmap.q, gmap.rgb)]
    if values is None:
        m64 = [a.astype(np.float64) for a in m32]
    else:
        m64 = [np.ascontiguousarray(a, np.float64) for a in values]
    return m32, m64


def project(gmap, cams, params: Params = Params()):
    """Dense [V, N] projection: visibility, depth key bits, tile rect and FP64 values."""
    lib = _load()
    (mo, su, q, rgb), (mo64, su64, q64, _) = _map(gmap)
    N, V = mo.shape[0], len(cams)
    cf, wh = _cams(cams, params)
    prm = params.block()
    out = dict(vis=np.zeros((V, N), np.int8), dkey=np.zeros((V, N), np.uint32), rect=np.zeros((V, N, 4), np.int32),
               mean2d=np.zeros((V, N, 2)), conic=np.zeros((V, N, 3)), cov2d=np.zeros((V, N, 3)),
               depth=np.zeros((V, N)), opac=np.zeros((V, N)))
    lib.or_project(N, _p(mo), _p(su), _p(q), _p(mo64), _p(su64), _p(q64), V, _p(cf), _p(wh), _p(prm),
                   _p(out["vis"]), _p(out["dkey"]), _p(out["rect"]), _p(out["mean2d"]), _p(out["conic"]),
                   _p(out["cov2d"]), _p(out["depth"]), _p(out["opac"]))
    return out


def all_pixels(cams, views=None) -> np.ndarray:
    views = range(len(cams)) if views is None else views
    chunks = []
    for v in views:
        W, H = cams[v].width, cams[v].height
        vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        chunks.append(np.stack([np.full(W * H, v), uu.ravel(), vv.ravel()], axis=1))
    return np.ascontiguousarray(np.concatenate(chunks), np.int32) if chunks else np.zeros((0, 3), np.int32)


def render(gmap, cams, params: Params = Params(), pixels=None, delta: float = 1e-3, values=None):
    """Brute-force compositing of the listed pixels (K x 3: view, u, v); all pixels if None.

    Returns dict with rgb [K,3], depth [K], unc [K], T [K], last_id [K], n_contrib [K],
    n_clamp [K], knife [K] (1 where a skip/stop decision lies within relative `delta`
    of its threshold).  `values` optionally overrides the FP64 parameter values
    (mo, su, q, rgb) while decisions keep using gmap's FP32 values.
    """
    lib = _load()
    (mo, su, q, rgb), (mo64, su64, q64, rgb64) = _map(gmap, values)
    pix = all_pixels(cams) if pixels is None else np.ascontiguousarray(pixels, np.int32)
    K = pix.shape[0]
    cf, wh = _cams(cams, params)
    prm = params.block()
    out = np.zeros((K, 5))
    T = np.zeros(K)
    last = np.zeros(K, np.int64)
    nc = np.zeros(K, np.int32)
    ncl = np.zeros(K, np.int32)
    kn = np.zeros(K, np.int8)
    lib.or_render(mo.shape[0], _p(mo), _p(su), _p(q), _p(mo64), _p(su64), _p(q64), _p(rgb64), len(cams), _p(cf),
                  _p(wh), _p(prm), K, _p(pix), float(delta), _p(out), _p(T), _p(last), _p(nc), _p(ncl), _p(kn))
    return dict(rgb=out[:, :3], depth=out[:, 3], unc=out[:, 4], T=T, last_id=last, n_contrib=nc, n_clamp=ncl,
                knife=kn.astype(bool), pixels=pix)


def render_images(gmap, cams, params: Params = Params(), delta: float = 1e-3, values=None):
    """Full images per view: list of dicts with [H, W(, 3)] arrays."""
    r = render(gmap, cams, params, None, delta, values)
    res, off = [], 0
    for c in cams:
        n = c.width * c.height
        sl = slice(off, off + n)
        shp = (c.height, c.width)
        res.append(dict(rgb=r["rgb"][sl].reshape(shp + (3,)), depth=r["depth"][sl].reshape(shp),
                        unc=r["unc"][sl].reshape(shp), T=r["T"][sl].reshape(shp),
                        last_id=r["last_id"][sl].reshape(shp), n_contrib=r["n_contrib"][sl].reshape(shp),
                        n_clamp=r["n_clamp"][sl].reshape(shp), knife=r["knife"][sl].reshape(shp)))
        off += n
    return res


def info_gain(gmap, cams, params: Params = Params()):
    """Per-view mean of the composited uncertainty channel, and the images it came from."""
    imgs = render_images(gmap, cams, params)
    return np.array([im["unc"].mean() for im in imgs]), imgs


def grad(gmap, cams, dimg, params: Params = Params(), values=None, want_2d: bool = False):
    """Analytic FP64 gradient of L = sum_views sum_pixels <dimg, (R, G, B, depth)>.

    dimg: list (one per view) of [H, W, 4] arrays.  Only pixels with a non-zero
    image gradient are visited.  Returns dict of [N, 4] arrays dmo (mu, logit),
    dsu (log-scales, 0), dq (quaternion), drgb (colour, 0) and, if want_2d,
    g2d [V, N, 8] = (dmean_x, dmean_y, dconic_a, dconic_b, dconic_c, dopacity,
    ddepth, 0) per view.
    """
    pix, gp = [], []
    for v, d in enumerate(dimg):
        d = np.asarray(d, np.float64)
        ys, xs = np.nonzero(np.any(d != 0, axis=2))
        pix.append(np.stack([np.full(len(xs), v), xs, ys], 1))
        gp.append(d[ys, xs])
    return grad_pixels(gmap, cams, np.concatenate(pix), np.concatenate(gp), params, values, want_2d)


def grad_pixels(gmap, cams, pixels, gpix, params: Params = Params(), values=None, want_2d: bool = False):
    """As `grad`, for an explicit list of pixels (K x 3: view, u, v) with gradients gpix (K x 4)."""
    lib = _load()
    (mo, su, q, rgb), (mo64, su64, q64, rgb64) = _map(gmap, values)
    N = mo.shape[0]
    cf, wh = _cams(cams, params)
    prm = params.block()
    pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 3)
    gp = np.ascontiguousarray(gpix, np.float64).reshape(-1, 4)
    out = {k: np.zeros((N, 4)) for k in ("dmo", "dsu", "dq", "drgb")}
    g2d = np.zeros((len(cams), N, 8)) if want_2d else None
    lib.or_grad(N, _p(mo), _p(su), _p(q), _p(mo64), _p(su64), _p(q64), _p(rgb64), len(cams), _p(cf), _p(wh),
                _p(prm), pix.shape[0], _p(pix), _p(gp), _p(out["dmo"]), _p(out["dsu"]), _p(out["dq"]),
                _p(out["drgb"]), _p(g2d) if want_2d else None)
    if want_2d:
        out["g2d"] = g2d
    return out


def tile_grid(cams, params: Params = Params()):
    """tiles_x per view and global tile base offsets (length V+1), with each view's tile size."""
    tx = np.array([-(-c.width // view_tile(c, params)[0]) for c in cams], np.int32)
    ty = np.array([-(-c.height // view_tile(c, params)[1]) for c in cams], np.int32)
    base = np.zeros(len(cams) + 1, np.int64)
    base[1:] = np.cumsum(tx.astype(np.int64) * ty)
    return tx, base


def records_from_projection(proj):
    """Visible (view, gaussian) entries as records in (gaussian id, view) order."""
    vis = proj["vis"].astype(bool)           # [V, N]
    g_idx, v_idx = np.nonzero(vis.T)          # row-major over (N, V): gaussian-major
    return dict(gid=g_idx.astype(np.uint32), view=v_idx.astype(np.uint32),
                rect=np.ascontiguousarray(proj["rect"][v_idx, g_idx]).astype(np.int32),
                dkey=np.ascontiguousarray(proj["dkey"][v_idx, g_idx]).astype(np.uint32))


def bin_sort(records, cams, params: Params = Params()):
    """Sorted pair list: keys u64 ((global tile << 32) | depth bits), vals (record index), ranges [T, 2]."""
    lib = _load()
    view = np.ascontiguousarray(records["view"], np.uint32)
    rect = np.ascontiguousarray(records["rect"], np.int32)
    dkey = np.ascontiguousarray(records["dkey"], np.uint32)
    R = view.shape[0]
    tx, base = tile_grid(cams, params)
    total = int(base[-1])
    P = int(lib.or_bin_count(R, _p(rect)))
    keys = np.zeros(P, np.uint64)
    vals = np.zeros(P, np.uint32)
    ranges = np.zeros((total, 2), np.int64)
    lib.or_bin(R, _p(view), _p(rect), _p(dkey), _p(tx), _p(base), total, _p(keys), _p(vals), _p(ranges))
    return dict(keys=keys, vals=vals, ranges=ranges, n_pairs=P, tile_base=base, tiles_x=tx)


def ex32(x: float) -> np.float32:
    return np.float32(_load().ex32(float(x)))


def lg32(x: float) -> np.float32:
    return np.float32(_load().lg32(float(x)))


# ------------------------------------------------------------------ render-free utility
def uncertainty_update(mo_prev: np.ndarray, mo_cur: np.ndarray, u_prev: np.ndarray, squared: bool = False):
    """Sec. IV-A: u_i = |mu_cur,i - mu_prev,i| in FP64 (squared for the ablation), for the
    Gaussians whose mean changed; the others keep u_prev (the paper's bookkeeping)."""
    d = mo_cur[:, :3].astype(np.float64) - mo_prev[:, :3].astype(np.float64)
    moved = (mo_cur[:, :3] != mo_prev[:, :3]).any(axis=1)
    d2 = (d * d).sum(axis=1)
    u = np.array(u_prev, np.float64, copy=True)
    u[moved] = d2[moved] if squared else np.sqrt(d2[moved])
    return u


def uncertainty_thresholds(mo: np.ndarray, u: np.ndarray, ground_z: float = -np.inf):
    """Mean and population standard deviation of u over the Gaussians with mu_z >= ground_z
    (exactly rounded FP64 sums), and the thresholds mean + sigma/2 (high) and mean - sigma/2
    (low).  Returns (mean, sigma, t_high, t_low, count)."""
    import math
    keep = mo[:, 2] >= np.float32(ground_z)
    x = u[keep].astype(np.float64)
    m = len(x)
    if m == 0:
        return 0.0, 0.0, 0.0, 0.0, 0
    mean = math.fsum(x) / m
    sigma = math.sqrt(math.fsum((x - mean) ** 2) / m)
    return mean, sigma, mean + 0.5 * sigma, mean - 0.5 * sigma, m


def visibility(mo: np.ndarray, cam, near_plane: float = 0.2, range_m: float = 5.0) -> np.ndarray:
    """v(x, g) of every mean for one camera, decided in FP32: t = R^T (mu - T) with each
    product and sum rounded to float32 in the order (R0 dx + R3 dy) + R6 dz (t_y, t_z
    likewise), pixel (fx t_x / t_z + cx, fy t_y / t_z + cy); visible iff
    near < t_z <= range and the pixel lies in [0, W) x [0, H)."""
    f = np.float32
    R = np.asarray(cam.R, np.float32).reshape(3, 3)
    T = np.asarray(cam.T, np.float32).reshape(3)
    dx = mo[:, 0].astype(f) - T[0]
    dy = mo[:, 1].astype(f) - T[1]
    dz = mo[:, 2].astype(f) - T[2]
    # t_j = sum_i R[i][j] d_i  (t = R^T d); R row-major: R[i][j] = R_flat[3 i + j]
    tx = (R[0, 0] * dx + R[1, 0] * dy) + R[2, 0] * dz
    ty = (R[0, 1] * dx + R[1, 1] * dy) + R[2, 1] * dz
    tz = (R[0, 2] * dx + R[1, 2] * dy) + R[2, 2] * dz
    with np.errstate(divide="ignore", invalid="ignore"):
        px = (f(cam.fx) * tx) / tz + f(cam.cx)
        py = (f(cam.fy) * ty) / tz + f(cam.cy)
    ok = (tz > f(near_plane)) & (tz <= f(range_m))
    return ok & (px >= 0) & (px < f(cam.width)) & (py >= 0) & (py < f(cam.height))


def view_utility(mo: np.ndarray, u: np.ndarray, cams, near_plane: float = 0.2, range_m: float = 5.0,
                 lam: float = 1.0, ground_z: float = -np.inf, mode: str = "xi", thresholds=None):
    """Eq. view_util per camera: xi = |visible G_H| - lam |visible G_L| (mode "xi", also
    returning the counts [V, 2]) or the FP64 sum of u over the visible Gaussians (mode
    "sum").  G_H = {u > t_high}, G_L = {u < t_low} from uncertainty_thresholds unless given."""
    keep = mo[:, 2] >= np.float32(ground_z)
    if thresholds is None:
        thresholds = uncertainty_thresholds(mo, u, ground_z)
    t_hi, t_lo = thresholds[2], thresholds[3]
    u64 = u.astype(np.float64)
    hi = keep & (u64 > t_hi)
    lo = keep & (u64 < t_lo)
    xi = np.zeros(len(cams))
    counts = np.zeros((len(cams), 2), np.int64)
    for v, cam in enumerate(cams):
        vis = visibility(mo, cam, near_plane, range_m)
        if mode == "sum":
            xi[v] = u64[vis & keep].sum()
        else:
            counts[v] = ((vis & hi).sum(), (vis & lo).sum())
            xi[v] = counts[v, 0] - lam * counts[v, 1]
    return xi, counts


def region_uncertainty(mo: np.ndarray, u: np.ndarray, origin, size: float, dims):
    """Mean u per cuboid region: region index (iz dims[1] + iy) dims[0] + ix with
    i = floor((mu - origin) / size) computed in float32 (the kernel's precision);
    Gaussians outside the grid are left out.  Returns (mean [R], count [R])."""
    f = np.float32
    idx = np.floor((mo[:, :3].astype(f) - np.asarray(origin, f)) / f(size))
    dims = np.asarray(dims, np.int64)
    inside = ((idx >= 0) & (idx < dims[None, :].astype(f))).all(axis=1)
    ii = idx[inside].astype(np.int64)
    r = (ii[:, 2] * dims[1] + ii[:, 1]) * dims[0] + ii[:, 0]
    R = int(dims.prod())
    cnt = np.bincount(r, minlength=R)
    tot = np.bincount(r, weights=u[inside].astype(np.float64), minlength=R)
    mean = np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)
    return mean, cnt


def trajectory_utility(mo: np.ndarray, u: np.ndarray, cams, n_traj: int, n_states: int, **kw):
    """Eq. traj_utility: per trajectory the sum over its states (cams[t * n_states + l]) of
    view_utility, and the first trajectory with the largest sum."""
    xi, _ = view_utility(mo, u, cams, **kw)
    s = xi.reshape(n_traj, n_states).sum(axis=1)
    return s, int(np.argmax(s))


def ex32v(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    _load().or_ex32v(x.size, _p(x), _p(y))
    return y


def collision_check(mo: np.ndarray, su: np.ndarray, points: np.ndarray, r_robot: float, lambda_g: float = 3.0,
                    ground_z: float = -np.inf):
    """Sec. IV-B collision checking: for every test point, the smallest |p - mu_i| - gamma_i
    (FP64) over the Gaussians with mu_z >= ground_z, gamma_i = r_robot + lambda_g r_i with
    r_i = exp(largest log-scale), and whether some |p - mu_i|^2 < gamma_i^2 -- decided in
    float32 like the kernel: d = p - mu, |d|^2 = (dx dx + dy dy) + dz dz, gamma = r_robot +
    lambda_g r, r from ex32.  Returns (margin [M], collides [M])."""
    f = np.float32
    keep = mo[:, 2] >= f(ground_z)
    mu = mo[keep, :3].astype(f)
    r = ex32v(su[keep, :3].max(axis=1))
    gam = f(r_robot) + f(lambda_g) * r
    gam2 = gam * gam
    gam64 = gam.astype(np.float64)
    margin = np.full(len(points), np.inf)
    hit = np.zeros(len(points), bool)
    for k, p in enumerate(np.asarray(points, f)[:, :3]):
        d = p[None, :] - mu
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        hit[k] = bool((d2 < gam2).any())
        if len(mu):
            exact = np.sqrt(((p.astype(np.float64)[None, :] - mu.astype(np.float64)) ** 2).sum(axis=1))
            margin[k] = (exact - gam64).min()
    return margin, hit


# ------------------------------------------------------------------ mapping loss (Eq. 3)
SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2


def ssim_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    """Normalised 1D Gaussian window; the 2D window is its outer product."""
    k = np.arange(size, dtype=np.float64) - (size - 1) / 2
    g = np.exp(-k * k / (2 * sigma * sigma))
    return g / g.sum()


def blur(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Same-size correlation of a 2D image with the window outer(g, g), zero outside the image."""
    from scipy.signal import correlate2d
    return correlate2d(img, np.outer(g, g), mode="same", boundary="fill", fillvalue=0.0)


def ssim_map(x: np.ndarray, y: np.ndarray, g=None):
    """Per-pixel SSIM of two single-channel images (FP64):
    ((2 mu_x mu_y + C1)(2 s_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)) with the
    windowed means mu = G*x, variances G*x^2 - mu^2 and covariance G*(xy) - mu_x mu_y."""
    g = ssim_window() if g is None else g
    mx, my = blur(x, g), blur(y, g)
    sxx = blur(x * x, g) - mx * mx
    syy = blur(y * y, g) - my * my
    sxy = blur(x * y, g) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def mapping_loss(rgb, depth, rgb_ref, depth_ref, w_d: float = 1.0, w_c: float = 0.4, w_s: float = 0.1):
    """Eq. 3 for one view (rgb [3,H,W], depth [H,W]):
    L = (1/N_p) sum_p (w_d |d - d_ref| + w_c |c - c_ref|_1) + w_s (1 - SSIM(c, c_ref)),
    SSIM = mean over the three channels and all pixels of ssim_map.  Returns (L, dL/drgb,
    dL/ddepth) in FP64; sign(0) = 0 for the L1 terms.  The SSIM gradient follows the moments:
    with m1 = G*x, m2 = G*x^2, m12 = G*(x y), dS/dx = G*(dS/dm1) + 2 x G*(dS/dm2) + y G*(dS/dm12)
    (the window is symmetric, so the adjoint of the zero-padded correlation is itself)."""
    g = ssim_window()
    rgb = np.asarray(rgb, np.float64)
    rgb_ref = np.asarray(rgb_ref, np.float64)
    depth = np.asarray(depth, np.float64)
    depth_ref = np.asarray(depth_ref, np.float64)
    N = depth.shape[0] * depth.shape[1]
    dd = depth - depth_ref
    dc = rgb - rgb_ref
    loss = (w_d * np.abs(dd).sum() + w_c * np.abs(dc).sum()) / N
    g_depth = w_d * np.sign(dd) / N
    g_rgb = w_c * np.sign(dc) / N
    s_tot = 0.0
    for ch in range(3):
        x, y = rgb[ch], rgb_ref[ch]
        m1, my = blur(x, g), blur(y, g)
        m2, m12 = blur(x * x, g), blur(x * y, g)
        syy = blur(y * y, g) - my * my
        A1 = 2 * m1 * my + SSIM_C1
        A2 = 2 * (m12 - m1 * my) + SSIM_C2
        B1 = m1 * m1 + my * my + SSIM_C1
        B2 = m2 - m1 * m1 + syy + SSIM_C2
        S = A1 * A2 / (B1 * B2)
        s_tot += S.sum()
        dm1 = 2 * my * (A2 - A1) / (B1 * B2) - 2 * m1 * S * (1 / B1 - 1 / B2)
        dm2 = -S / B2
        dm12 = 2 * A1 / (B1 * B2)
        dS = blur(dm1, g) + 2 * x * blur(dm2, g) + y * blur(dm12, g)
        g_rgb[ch] -= w_s * dS / (3 * N)
    loss += w_s * (1 - s_tot / (3 * N))
    return loss, g_rgb, g_depth


def mapping_loss_views(rgbs, depths, rgb_refs, depth_refs, w_d: float = 1.0, w_c: float = 0.4, w_s: float = 0.1):
    """Eq. 3 over several views with N_p = the total pixel count of all views (each view is its
    own image for SSIM): L = sum_v (N_v / N_p) L_v, and each view's gradient scaled by N_v / N_p.
    Returns (L, mean |d - d_ref|, mean |c - c_ref|_1, SSIM, [dL/drgb_v], [dL/ddepth_v])."""
    n_v = [np.asarray(d).size for d in depths]
    n_p = float(sum(n_v))
    L, l1d, l1c, ss, g_rgb, g_depth = 0.0, 0.0, 0.0, 0.0, [], []
    for x, d, y, dr, n in zip(rgbs, depths, rgb_refs, depth_refs, n_v):
        Lv, gr, gd = mapping_loss(x, d, y, dr, w_d, w_c, w_s)
        f = n / n_p
        L += f * Lv
        l1d += np.abs(np.asarray(d, np.float64) - np.asarray(dr, np.float64)).sum() / n_p
        l1c += np.abs(np.asarray(x, np.float64) - np.asarray(y, np.float64)).sum() / n_p
        ss += sum(ssim_map(np.asarray(x[c], np.float64), np.asarray(y[c], np.float64)).sum() for c in range(3)) / (3 * n_p)
        g_rgb.append(f * gr)
        g_depth.append(f * gd)
    return L, l1d, l1c, ss, g_rgb, g_depth


# ------------------------------------------------------------------ optimiser of the mapping iterations
def adam_step(p, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba), the optimiser of the mapping iterations (the map is
    refined by gradient steps on the rendering loss, Eq. 2 / Sec. IV-A), in FP64:
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2, and with the bias corrections
    c1 = 1 - b1^t, c2 = 1 - b2^t: p <- p - (lr / c1) m / (sqrt(v) / sqrt(c2) + eps).
    t is the number of this step (1 for the first).  Returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    c1, c2 = 1.0 - beta1 ** t, 1.0 - beta2 ** t
    p = p - (lr / c1) * m / (np.sqrt(v) / math.sqrt(c2) + eps)
    return p, m, v
