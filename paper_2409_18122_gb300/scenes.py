"""Seeded synthetic inputs: Gaussian maps and camera sets.

This module only draws random numbers and lays them out; it contains none of
the splatting arithmetic (no projection, compositing or sorting).  Both the
CUDA path and the FP64 oracle are fed from here, so neither depends on the
other for its inputs.

The paper's own workloads (iTHOR rooms, MP3D scenes, onboard maps) are not
available; these generators stand in for them with the shapes and value
distributions of the paper's setting: a map of Gaussians parameterised by
colour, position, size and opacity (Sec. III, "Gaussian Splatting") plus the
per-Gaussian uncertainty channel u_i = |mu_k - mu_{k-1}| (Sec. IV-A), and
pinhole cameras posed by a rotation R_k and translation T_k in the world frame.

Map layout (float32, four arrays of shape [N, 4]):
  mo  = (mu_x, mu_y, mu_z, opacity_logit)
  su  = (log_scale_0, log_scale_1, log_scale_2, u)
  q   = (w, x, y, z)            unnormalised rotation quaternion
  rgb = (r, g, b, 0)

Camera: fx, fy, cx, cy, width, height, R (3x3, camera-to-world, row-major,
OpenCV axes: x right, y down, z forward), T (camera centre in world).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))
    T: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))
    tile_w: int = 0        # this view's screen tile; 0 = the renderer's default
    tile_h: int = 0

    def __post_init__(self):
        self.R = np.asarray(self.R, dtype=np.float32).reshape(3, 3)
        self.T = np.asarray(self.T, dtype=np.float32).reshape(3)
        self.fx, self.fy = float(np.float32(self.fx)), float(np.float32(self.fy))
        self.cx, self.cy = float(np.float32(self.cx)), float(np.float32(self.cy))
        self.width, self.height = int(self.width), int(self.height)

    @property
    def n_pixels(self) -> int:
        return self.width * self.height

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """The same camera restricted to the pixel window [x0, x0+w) x [y0, y0+h).

        Pixel (u, v) of the crop samples the same ray as pixel (u+x0, v+y0) of
        the full image, so a crop renders exactly that window.
        """
        return Camera(self.fx, self.fy, self.cx - x0, self.cy - y0, w, h, self.R.copy(), self.T.copy(),
                      self.tile_w, self.tile_h)

    def with_tile(self, tile_w: int, tile_h: int) -> "Camera":
        """The same camera rendered with its own screen tile size."""
        return Camera(self.fx, self.fy, self.cx, self.cy, self.width, self.height, self.R.copy(), self.T.copy(),
                      tile_w, tile_h)


@dataclass
class GaussianMap:
    mo: np.ndarray
    su: np.ndarray
    q: np.ndarray
    rgb: np.ndarray

    def __post_init__(self):
        for k in ("mo", "su", "q", "rgb"):
            a = np.ascontiguousarray(getattr(self, k), dtype=np.float32)
            assert a.ndim == 2 and a.shape[1] == 4, k
            setattr(self, k, a)
        n = self.mo.shape[0]
        assert self.su.shape[0] == n and self.q.shape[0] == n and self.rgb.shape[0] == n

    @property
    def n(self) -> int:
        return int(self.mo.shape[0])

    def subset(self, idx) -> "GaussianMap":
        idx = np.asarray(idx)
        return GaussianMap(self.mo[idx], self.su[idx], self.q[idx], self.rgb[idx])

    def copy(self) -> "GaussianMap":
        return GaussianMap(self.mo.copy(), self.su.copy(), self.q.copy(), self.rgb.copy())

    def arrays(self):
        return self.mo, self.su, self.q, self.rgb


@dataclass
class Scene:
    name: str
    gmap: GaussianMap
    cams: List[Camera]
    seed: int


# ----------------------------------------------------------------------------
# parameter draws shared by all configurations
# ----------------------------------------------------------------------------

def _attributes(rng: np.random.Generator, n: int):
    ls = rng.normal(-3.0, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit = rng.normal(0.0, 1.0, size=n)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    u = rng.uniform(0.0, 1.0, size=n)
    return ls, q, logit, rgb, u


def _pack(mu, ls, q, logit, rgb, u) -> GaussianMap:
    n = mu.shape[0]
    mo = np.empty((n, 4), np.float32)
    mo[:, :3] = mu
    mo[:, 3] = logit
    su = np.empty((n, 4), np.float32)
    su[:, :3] = ls
    su[:, 3] = u
    rgbp = np.zeros((n, 4), np.float32)
    rgbp[:, :3] = rgb
    return GaussianMap(mo, su, q.astype(np.float32), rgbp)


def yaw_camera(x: float, y: float, z: float, yaw: float, width: int, height: int,
               f: float, cx: float | None = None, cy: float | None = None) -> Camera:
    """A level camera at (x, y, z) looking horizontally along heading `yaw`.

    Forward z_c = (cos yaw, sin yaw, 0), down y_c = (0, 0, -1) (world z is up),
    right x_c = y_c x z_c.  R has these as columns (camera-to-world).
    """
    zc = np.array([np.cos(yaw), np.sin(yaw), 0.0])
    yc = np.array([0.0, 0.0, -1.0])
    xc = np.cross(yc, zc)
    R = np.stack([xc, yc, zc], axis=1)
    return Camera(f, f, width / 2.0 if cx is None else cx, height / 2.0 if cy is None else cy,
                  width, height, R, np.array([x, y, z]))


def room_means(rng: np.random.Generator, n: int, extent=(10.0, 10.0, 3.0), n_patches: int = 50,
               side=(0.5, 2.0), sigma_off: float = 0.02) -> np.ndarray:
    """Means clustered on random square planar patches inside a box room.

    Patch centre uniform in the room, normal uniform on the sphere, side length
    uniform in `side`, points uniform on the square plus N(0, sigma_off) along
    the normal.  Gaussians are split evenly across patches (remainder to the
    first ones).
    """
    ext = np.asarray(extent, dtype=np.float64)
    centres = rng.uniform(0.0, 1.0, size=(n_patches, 3)) * ext
    normals = rng.normal(size=(n_patches, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    sides = rng.uniform(side[0], side[1], size=n_patches)
    # in-plane basis per patch
    helper = np.where(np.abs(normals[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    e1 = np.cross(normals, helper)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(normals, e1)
    counts = np.full(n_patches, n // n_patches)
    counts[: n % n_patches] += 1
    pid = np.repeat(np.arange(n_patches), counts)
    a = (rng.uniform(size=n) - 0.5) * sides[pid]
    b = (rng.uniform(size=n) - 0.5) * sides[pid]
    off = rng.normal(0.0, sigma_off, size=n)
    return centres[pid] + a[:, None] * e1[pid] + b[:, None] * e2[pid] + off[:, None] * normals[pid]


# ----------------------------------------------------------------------------
# the five workload configurations
# ----------------------------------------------------------------------------

def config0(seed: int = 1000) -> Scene:
    """2,000 Gaussians uniform in [-2,2]^2 x [1,5]; one 128x96 view at the origin looking +z."""
    rng = np.random.default_rng(seed)
    n = 2000
    mu = rng.uniform([-2.0, -2.0, 1.0], [2.0, 2.0, 5.0], size=(n, 3))
    g = _pack(mu, *_attributes(rng, n))
    cam = Camera(100.0, 100.0, 64.0, 48.0, 128, 96)
    return Scene("cfg0", g, [cam], seed)


def _room_pose(rng, extent: float = 10.0):
    """Keyframe pose: position uniform in the room (0.5 m from the walls), height
    U[1, 2] m, heading towards the room centre plus U(-45, 45) degrees, so that a
    mapping keyframe looks into the mapped space rather than at a nearby wall."""
    x, y = rng.uniform(0.5, extent - 0.5, size=2)
    z = rng.uniform(1.0, 2.0)
    c = extent / 2.0
    yaw = np.arctan2(c - y, c - x) + rng.uniform(-np.pi / 4, np.pi / 4)
    return x, y, z, yaw


def config1(seed: int = 1001, n: int = 200_000) -> Scene:
    """200,000 Gaussians on 50 patches in a 10x10x3 m room; one 640x480 view, f=525."""
    rng = np.random.default_rng(seed)
    mu = room_means(rng, n)
    g = _pack(mu, *_attributes(rng, n))
    cam = yaw_camera(*_room_pose(rng), 640, 480, 525.0)
    return Scene("cfg1", g, [cam], seed)


def config2(seed: int = 1002, n: int = 500_000, n_views: int = 4, width: int = 640, height: int = 480,
            f: float = 525.0) -> Scene:
    """500,000 room Gaussians; 4 keyframes at 640x480 posed as in config 1."""
    rng = np.random.default_rng(seed)
    mu = room_means(rng, n)
    g = _pack(mu, *_attributes(rng, n))
    cams = [yaw_camera(*_room_pose(rng), width, height, f) for _ in range(n_views)]
    return Scene("cfg2", g, cams, seed)


IG_RESOLUTIONS = ((80, 60), (160, 120), (320, 240))


def candidate_lattice(rng, n_side: int, extent: float, resolutions, z: float = 1.5):
    """Candidate poses on an n_side x n_side lattice at height z with random yaw.

    View i gets resolutions[i % len(resolutions)]; focal length f = 0.8203 W
    (the horizontal field of view of a 640-wide, f=525 camera).
    """
    xs = np.linspace(0.5, extent - 0.5, n_side)
    cams = []
    i = 0
    for y in xs:
        for x in xs:
            w, h = resolutions[i % len(resolutions)]
            yaw = rng.uniform(0.0, 2 * np.pi)
            cams.append(yaw_camera(x, y, z, yaw, w, h, 0.8203 * w))
            i += 1
    return cams


def config3(seed: int = 1003, n: int = 1_000_000, n_side: int = 16) -> Scene:
    """1,000,000 room Gaussians; 256 candidates, one third each at 80x60 / 160x120 / 320x240."""
    rng = np.random.default_rng(seed)
    mu = room_means(rng, n)
    g = _pack(mu, *_attributes(rng, n))
    cams = candidate_lattice(rng, n_side, 10.0, IG_RESOLUTIONS)
    return Scene("cfg3", g, cams, seed)


def config4(seed: int = 1004, n: int = 3_000_000):
    """40x40x3 m map, ~750 patches, 3M Gaussians; 8 keyframes 1280x720 (f=1050) and
    1,024 candidates on a 32x32 lattice, half 160x120 and half 320x240."""
    rng = np.random.default_rng(seed)
    mu = room_means(rng, n, extent=(40.0, 40.0, 3.0), n_patches=750)
    g = _pack(mu, *_attributes(rng, n))
    keys = [yaw_camera(*_room_pose(rng, 40.0), 1280, 720, 1050.0) for _ in range(8)]
    cands = candidate_lattice(rng, 32, 40.0, ((160, 120), (320, 240)))
    return Scene("cfg4", g, keys, seed), cands


def perturbed(g: GaussianMap, seed: int, sigma_mu: float = 0.01, sigma_rgb: float = 0.05) -> GaussianMap:
    """Copy of a map with means + N(0, sigma_mu) and colours + N(0, sigma_rgb) (mapping targets)."""
    rng = np.random.default_rng(seed)
    h = g.copy()
    h.mo[:, :3] += rng.normal(0.0, sigma_mu, size=(g.n, 3)).astype(np.float32)
    h.rgb[:, :3] += rng.normal(0.0, sigma_rgb, size=(g.n, 3)).astype(np.float32)
    return h


def random_scene(seed: int, n: int, cams: Sequence[Camera], box=((-2, -2, 1), (2, 2, 5)),
                 log_scale=(-3.0, 0.5)) -> GaussianMap:
    """Uniform means in an axis-aligned box with the standard attribute draws."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(box[0], box[1], size=(n, 3))
    ls, q, logit, rgb, u = _attributes(rng, n)
    ls = rng.normal(log_scale[0], log_scale[1], size=(n, 3))
    return _pack(mu, ls, q, logit, rgb, u)


def synthetic_records(seed: int, n_gauss: int, cams: Sequence[Camera], tile_w: int = 16, tile_h: int = 16,
                      p_visible: float = 0.5, max_extent: int = 6, tie_frac: float = 0.1):
    """Random projection records for exercising binning and sorting alone.

    Returns dict with per-record arrays in (view, gaussian id) order (the
    records of a view contiguous, as the projection writes them): gid (u32),
    view (u32), rect (int32 [R,4] = tile x0, y0, x1, y1 with exclusive ends)
    and depth (float32 > 0).  A fraction `tie_frac` of the depths are copied
    from another record so that equal keys occur.
    """
    rng = np.random.default_rng(seed)
    gids, views, rects, depths = [], [], [], []
    for g in range(n_gauss):
        for v, cam in enumerate(cams):
            if rng.uniform() >= p_visible:
                continue
            tx = -(-cam.width // tile_w)
            ty = -(-cam.height // tile_h)
            w = int(rng.integers(1, min(max_extent, tx) + 1))
            h = int(rng.integers(1, min(max_extent, ty) + 1))
            x0 = int(rng.integers(0, tx - w + 1))
            y0 = int(rng.integers(0, ty - h + 1))
            gids.append(g)
            views.append(v)
            rects.append((x0, y0, x0 + w, y0 + h))
            depths.append(rng.uniform(0.2, 12.0))
    depth = np.asarray(depths, np.float32)
    r = len(depth)
    if r > 1 and tie_frac > 0:
        k = int(tie_frac * r)
        dst = rng.integers(0, r, size=k)
        src = rng.integers(0, r, size=k)
        depth[dst] = depth[src]
    view = np.asarray(views, np.uint32)
    order = np.argsort(view, kind="stable")
    return dict(gid=np.asarray(gids, np.uint32)[order], view=view[order],
                rect=np.asarray(rects, np.int32).reshape(-1, 4)[order], depth=depth[order])
