"""PyTorch front end of libgs103.so: device buffers, streams, autograd.

Every step of the splatting path runs in the library's CUDA kernels; this
module only allocates tensors (PyTorch owns all device memory), passes their
pointers and the current stream through the C ABI, and wraps the forward and
backward entry points in a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

CAMERA_DTYPE = np.dtype([("fx", "<f4"), ("fy", "<f4"), ("cx", "<f4"), ("cy", "<f4"), ("width", "<i4"),
                         ("height", "<i4"), ("R", "<f4", (9,)), ("T", "<f4", (3,)), ("tile_w", "<i4"),
                         ("tile_h", "<i4")])
assert CAMERA_DTYPE.itemsize == 80


@dataclass
class RenderParams:
    """Rendering constants the paper leaves unstated (see include/gs.h gs_params)."""
    tile_w: int = 16
    tile_h: int = 16
    eps2d: float = 0.3
    near: float = 0.2
    guard: float = 1.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    ig_batch: int = 0      # chunk depth of the information-gain compositing: 4, 8 or 16 (0: 8)
    fwd_batch: int = 0     # chunk depth of the forward compositing: 1, 2 or 4 (0: 2)

    def c(self) -> L.gs_params:
        return L.gs_params(self.tile_w, self.tile_h, self.eps2d, self.near, self.guard, self.alpha_min,
                           self.alpha_max, self.T_min, self.ig_batch, self.fwd_batch)


class StageTimer:
    """Optional CUDA-event bracketing of every C-ABI call (for measurement only).

    When `gs.TIMER` is a StageTimer, each entry point call records a start and
    an end event on the stream it is launched on; `durations_ms(name)` returns
    the per-call device times after a synchronise.
    """

    def __init__(self):
        self.events = {}

    def bracket(self, name, stream):
        s = torch.cuda.current_stream() if stream is None else stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        self.events.setdefault(name, []).append((e0, e1))
        return s, e0, e1

    def durations_ms(self, name):
        return [a.elapsed_time(b) for a, b in self.events.get(name, [])]

    def clear(self):
        self.events = {}


TIMER: Optional[StageTimer] = None


def _timed(name, stream, fn):
    if TIMER is None:
        return fn()
    s, e0, e1 = TIMER.bracket(name, stream)
    e0.record(s)
    r = fn()
    e1.record(s)
    return r


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def pack_cameras(cams) -> np.ndarray:
    """Cameras (objects with fx, fy, cx, cy, width, height, R, T) -> gs_camera records."""
    a = np.zeros(len(cams), CAMERA_DTYPE)
    for i, c in enumerate(cams):
        a[i] = (c.fx, c.fy, c.cx, c.cy, c.width, c.height, np.asarray(c.R, np.float32).reshape(9),
                np.asarray(c.T, np.float32).reshape(3), getattr(c, "tile_w", 0), getattr(c, "tile_h", 0))
    return a


def cameras_to_device(cams, device="cuda") -> torch.Tensor:
    return torch.from_numpy(pack_cameras(cams).view(np.uint8).copy()).to(device)


def view_tile(c, params: RenderParams):
    """Tile size of a view: the camera's own (tile_w, tile_h, if non-zero) else the params'."""
    tw, th = getattr(c, "tile_w", 0), getattr(c, "tile_h", 0)
    return (tw, th) if tw and th else (params.tile_w, params.tile_h)


def valid_tile(tw: int, th: int) -> bool:
    """The tile sizes the kernels accept (include/gs.h gs_params)."""
    return tw in (8, 16, 32, 64) and th >= 8 and th % 8 == 0 and tw * th in (64, 128, 256, 512, 1024)


def camera_ok(c, params: RenderParams) -> bool:
    """The library's camera check (a camera failing it sets GS_FLAG_BAD_CAMERA and gets no tiles):
    a positive image size, positive finite focal lengths and a valid tile size."""
    tw, th = view_tile(c, params)
    fx, fy = float(np.float32(c.fx)), float(np.float32(c.fy))
    return (c.width > 0 and c.height > 0 and fx > 0 and fy > 0 and np.isfinite(fx) and np.isfinite(fy)
            and valid_tile(tw, th))


def tile_grid(cams, params: RenderParams):
    """Per view: tiles_x, tiles_y; and the tile and pixel offsets of the views (length V+1).
    A view whose camera fails camera_ok has no tiles but keeps its W x H pixels."""
    ok = [camera_ok(c, params) for c in cams]
    tx = np.array([-(-c.width // view_tile(c, params)[0]) if k else 0 for c, k in zip(cams, ok)], np.int64)
    ty = np.array([-(-c.height // view_tile(c, params)[1]) if k else 0 for c, k in zip(cams, ok)], np.int64)
    tiles = tx * ty
    pix = np.array([max(c.width, 0) * max(c.height, 0) for c in cams], np.int64)
    tile_base = np.concatenate([[0], np.cumsum(tiles)])
    pix_base = np.concatenate([[0], np.cumsum(pix)])
    return tx, ty, tile_base, pix_base


class GaussianMapTensors:
    """The four [N, 4] float32 device arrays of include/gs.h gs_map."""

    def __init__(self, mo: torch.Tensor, su: torch.Tensor, q: torch.Tensor, rgb: torch.Tensor):
        self.mo, self.su, self.q, self.rgb = mo, su, q, rgb

    @staticmethod
    def from_numpy(g, device="cuda") -> "GaussianMapTensors":
        return GaussianMapTensors(*(torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in
                                    (g.mo, g.su, g.q, g.rgb)))

    @property
    def n(self) -> int:
        return int(self.mo.shape[0])

    def c(self) -> L.gs_map:
        return make_map(self.mo, self.su, self.q, self.rgb)


def make_map(mo, su, q, rgb) -> L.gs_map:
    for t in (mo, su, q, rgb):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.dim() != 2 or t.shape[1] != 4:
            raise ValueError("map arrays must be contiguous float32 CUDA tensors of shape [N, 4]")
    return L.gs_map(_ptr(mo), _ptr(su), _ptr(q), _ptr(rgb), int(mo.shape[0]))


def _require(t: Optional[torch.Tensor], what: str, numel: int, dtype=torch.float32):
    """Host-side check before a tensor's pointer crosses the C ABI: the library reads and writes
    device memory, so a host, non-contiguous, wrongly typed or too small tensor is refused here
    (None passes: the entry points take NULL for optional buffers)."""
    if t is None:
        return
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
            and t.numel() >= numel):
        raise ValueError("%s must be a contiguous %s CUDA tensor of at least %d elements" % (what, dtype, numel))


def _require_images(img, P: int):
    for k, n, dt in (("rgb", 3 * P, torch.float32), ("depth", P, torch.float32), ("unc", P, torch.float32),
                     ("T", P, torch.float32), ("last", P, torch.int32), ("n_contrib", P, torch.int32)):
        _require(img.get(k), "image " + k, n, dt)


def _alloc_u32(n, device):
    return torch.empty(max(int(n), 1), dtype=torch.int32, device=device)


class Frame:
    """Device buffers for projecting, binning and rendering one map into a fixed camera set.

    pair_capacity bounds the number of (tile, Gaussian) pairs; exceeding it sets
    GS_FLAG_PAIR_OVERFLOW (see `check_status` / `grow_if_needed`).  with_color=False
    leaves out the per-record colours (scoring only); with_pair_tiles=False leaves
    out the global tile id of every pair (compositing needs only the ranges);
    with_gid=False leaves out the Gaussian id of every record (the kernels never read it);
    with_view=False leaves out the view id of every record (binning then finds each view's
    records through the projection's group offsets).  with_item_order=False leaves out the
    binning's longest-list-first order of the warp items (the render kernels then take
    their items tile by tile; the outputs are the same).
    """

    def __init__(self, n: int, cams: Sequence, params: RenderParams = RenderParams(),
                 pair_capacity: Optional[int] = None, device="cuda", with_color: bool = True,
                 with_pair_tiles: bool = True, record_capacity: Optional[int] = None, with_gid: bool = True,
                 with_view: bool = True, with_item_order: bool = True):
        self.device = torch.device(device)
        self.with_item_order = with_item_order
        self.params = params
        self.with_color = with_color
        self.with_gid = with_gid
        self.with_view = with_view
        self.with_pair_tiles = with_pair_tiles
        self.cams = list(cams)
        self.V = len(self.cams)
        self.n = int(n)
        self.cams_dev = cameras_to_device(self.cams, self.device)
        self.tiles_x, self.tiles_y, self.tile_base, self.pix_base = tile_grid(self.cams, params)
        self.n_tiles = int(self.tile_base[-1])
        self.n_pixels = int(self.pix_base[-1])
        # warp items: 32-pixel blocks, tile_w * tile_h / 32 per tile
        self.n_items = 0
        for v in range(self.V):
            tw, th = self.view_tile(v)
            self.n_items += int(self.tiles_x[v] * self.tiles_y[v]) * tw * th // 32
        # records: at most n * V; a smaller capacity (large batches) grows on overflow
        self.rec_capacity = max(int(record_capacity) if record_capacity else self.n * self.V, 1)
        # bumped by every projection and binning: the backward pass replays the records and tile
        # lists of its own forward, so it refuses to run once they have been overwritten
        self.generation = 0
        if pair_capacity is None:
            pair_capacity = min(max(1 << 20, 8 * self.n * self.V), (1 << 31) - 1)
        self._alloc(int(pair_capacity))

    def _alloc(self, pair_capacity: int):
        d, rc = self.device, self.rec_capacity
        for name in ("pair_tile", "pair_rec", "ws", "splat", "color_d", "gid", "view", "rect"):
            if hasattr(self, name):
                setattr(self, name, None)   # release before reallocating
        self.pair_capacity = pair_capacity
        self.status = torch.zeros(1, dtype=torch.int32, device=d)
        self.rec_count = torch.zeros(1, dtype=torch.int32, device=d)
        self.view_info = torch.zeros(4 * (self.V + 1), dtype=torch.int32, device=d)
        self.gid = _alloc_u32(rc, d) if self.with_gid else None
        self.view = _alloc_u32(rc, d) if self.with_view else None
        self.splat = torch.empty((rc, 8), dtype=torch.float32, device=d)
        self.color_d = torch.empty((rc, 4), dtype=torch.float32, device=d) if self.with_color else None
        self.rect = torch.empty((rc, 4), dtype=torch.int16, device=d)
        self.depth_key = _alloc_u32(rc, d)
        self.n_slots = ((self.n + 31) // 32) * self.V
        self.grp_mask = _alloc_u32(self.n_slots, d)
        self.grp_base = _alloc_u32(self.n_slots + 1, d)
        self.pair_count = torch.zeros(1, dtype=torch.int32, device=d)
        self.pair_tile = _alloc_u32(pair_capacity, d) if self.with_pair_tiles else None
        self.pair_rec = _alloc_u32(pair_capacity, d)
        self.ranges = torch.zeros((max(self.n_tiles, 1), 2), dtype=torch.int32, device=d)
        self.item_order = _alloc_u32(self.n_items, d) if self.with_item_order else None
        ws = max(L.workspace_size(L.GS_OP_PROJECT, self.n, self.V),
                 L.workspace_size(L.GS_OP_BIN_SORT, self.n, self.V, rc, pair_capacity, max(self.n_tiles, 1)),
                 L.workspace_size(L.GS_OP_RENDER_BWD, self.n, self.V, rc))
        self.ws = torch.empty(max(ws, 256), dtype=torch.uint8, device=d)
        self.c_proj = L.gs_proj(rc, _ptr(self.rec_count), _ptr(self.status), _ptr(self.view_info), _ptr(self.gid),
                                _ptr(self.view), _ptr(self.splat), _ptr(self.color_d), _ptr(self.rect),
                                _ptr(self.depth_key), _ptr(self.grp_mask), _ptr(self.grp_base))
        self.c_bins = L.gs_bins(pair_capacity, max(self.n_tiles, 1), _ptr(self.pair_count), _ptr(self.pair_tile),
                                _ptr(self.pair_rec), _ptr(self.ranges), _ptr(self.item_order),
                                self.n_items if self.with_item_order else 0)
        self.c_params = self.params.c()

    def view_tile(self, v: int):
        return view_tile(self.cams[v], self.params)

    # -------------------------------------------------------------- stages
    def project(self, gmap: GaussianMapTensors, stream=None):
        if gmap.n != self.n:
            raise ValueError("map has %d Gaussians, frame was built for %d" % (gmap.n, self.n))
        m = gmap.c()
        self.generation += 1
        _timed("gs_project", stream, lambda: L.check(
            L.lib().gs_project(ctypes.byref(m), _ptr(self.cams_dev), self.V, ctypes.byref(self.c_params),
                               ctypes.byref(self.c_proj), _ptr(self.ws), self.ws.numel(), _stream(stream)),
            "gs_project"))

    def bin_sort(self, stream=None):
        self.generation += 1
        _timed("gs_bin_sort", stream, lambda: L.check(
            L.lib().gs_bin_sort(ctypes.byref(self.c_proj), _ptr(self.cams_dev), self.V, ctypes.byref(self.c_params),
                                ctypes.byref(self.c_bins), _ptr(self.ws), self.ws.numel(), _stream(stream)),
            "gs_bin_sort"))

    def new_images(self, with_rgb=True, with_depth=True, with_unc=True, with_counts=False):
        d, P = self.device, self.n_pixels
        return dict(rgb=torch.empty(3 * P, dtype=torch.float32, device=d) if with_rgb else None,
                    depth=torch.empty(P, dtype=torch.float32, device=d) if with_depth else None,
                    unc=torch.empty(P, dtype=torch.float32, device=d) if with_unc else None,
                    T=torch.empty(P, dtype=torch.float32, device=d),
                    last=torch.empty(P, dtype=torch.int32, device=d),
                    n_contrib=torch.empty(P, dtype=torch.int32, device=d) if with_counts else None)

    def render_fwd(self, gmap: GaussianMapTensors, images=None, stream=None):
        img = self.new_images() if images is None else images
        _require_images(img, self.n_pixels)
        c_img = L.gs_image(_ptr(img["rgb"]), _ptr(img["depth"]), _ptr(img["unc"]), _ptr(img["T"]),
                           _ptr(img["last"]), _ptr(img.get("n_contrib")))
        m = gmap.c()
        _timed("gs_render_fwd", stream, lambda: L.check(
            L.lib().gs_render_fwd(ctypes.byref(m), ctypes.byref(self.c_proj), ctypes.byref(self.c_bins),
                                  _ptr(self.cams_dev), self.V, ctypes.byref(self.c_params), ctypes.byref(c_img),
                                  _stream(stream)), "gs_render_fwd"))
        return img

    def render_bwd(self, gmap: GaussianMapTensors, images, d_rgb=None, d_depth=None, grads=None, stream=None):
        g = grads
        if g is None:
            g = {k: torch.empty((self.n, 4), dtype=torch.float32, device=self.device) for k in
                 ("dmo", "dsu", "dq", "drgb")}
        _require_images(images, self.n_pixels)
        _require(d_rgb, "d_rgb", 3 * self.n_pixels)
        _require(d_depth, "d_depth", self.n_pixels)
        for k in ("dmo", "dsu", "dq", "drgb"):
            _require(g[k], "gradient " + k, 4 * self.n)
        c_img = L.gs_image(_ptr(images["rgb"]), _ptr(images["depth"]), _ptr(images["unc"]), _ptr(images["T"]),
                           _ptr(images["last"]), None)
        c_g = L.gs_image_grad(_ptr(d_rgb), _ptr(d_depth))
        c_out = L.gs_map_grad(_ptr(g["dmo"]), _ptr(g["dsu"]), _ptr(g["dq"]), _ptr(g["drgb"]))
        m = gmap.c()
        _timed("gs_render_bwd", stream, lambda: L.check(
            L.lib().gs_render_bwd(ctypes.byref(m), ctypes.byref(self.c_proj), ctypes.byref(self.c_bins),
                                  ctypes.byref(c_img), ctypes.byref(c_g), _ptr(self.cams_dev), self.V,
                                  ctypes.byref(self.c_params), ctypes.byref(c_out), _ptr(self.ws), self.ws.numel(),
                                  _stream(stream)), "gs_render_bwd"))
        return g

    def info_gain(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Per-view mean of the composited uncertainty of the projected and binned views
        (gs_info_gain_composite; call project and bin_sort first)."""
        o = torch.zeros(self.V, dtype=torch.float32, device=self.device) if out is None else out
        _require(o, "out", self.V)
        if not hasattr(self, "ig_ws"):
            self.ig_ws = torch.empty(L.workspace_size(L.GS_OP_IG_COMPOSITE, self.n, self.V, 0, 0,
                                                      max(self.n_tiles, 1)), dtype=torch.uint8, device=self.device)
        _timed("gs_info_gain_composite", stream, lambda: L.check(
            L.lib().gs_info_gain_composite(ctypes.byref(self.c_proj), ctypes.byref(self.c_bins), _ptr(self.cams_dev),
                                           self.V, ctypes.byref(self.c_params), L.GS_IG_RENDER_MEAN, _ptr(o),
                                           _ptr(self.ig_ws), self.ig_ws.numel(), _stream(stream)),
            "gs_info_gain_composite"))
        return o

    def forward(self, gmap: GaussianMapTensors, images=None, stream=None):
        """project -> bin_sort -> render_fwd."""
        self.project(gmap, stream)
        self.bin_sort(stream)
        return self.render_fwd(gmap, images, stream)

    # -------------------------------------------------------------- status
    def reset_status(self):
        self.status.zero_()

    def read_status(self) -> int:
        flags = ctypes.c_uint32(0)
        L.lib().gs_read_status(_ptr(self.status), ctypes.byref(flags))
        return int(flags.value)

    def check_status(self):
        f = self.read_status()
        if f & L.GS_FLAG_ERROR_MASK:
            raise L.GSError("device status flags 0x%x (pairs %d / capacity %d)" %
                            (f, int(self.pair_count.item()) & 0xFFFFFFFF, self.pair_capacity))
        return f

    def grow_if_needed(self, margin: float = 1.25) -> bool:
        """After a synchronised forward: if records or pairs overflowed, reallocate with room for
        them (returns True; run the forward again)."""
        f = self.read_status()
        if f & L.GS_FLAG_RECORD_OVERFLOW:
            need = int(self.grp_base[self.n_slots].item()) & 0xFFFFFFFF
            self.rec_capacity = max(min(int(need * margin) + 1024, self.n * self.V), 1)
            self.status.zero_()
            self._alloc(self.pair_capacity)
            self.generation += 1
            return True
        if f & L.GS_FLAG_PAIR_OVERFLOW:
            need = int(self.pair_count.item()) & 0xFFFFFFFF
            if need == 0xFFFFFFFF:
                need = 2 * self.pair_capacity
            self._alloc(min(int(need * margin) + 1024, (1 << 32) - 2))
            self.generation += 1
            return True
        return False

    # -------------------------------------------------------------- views of the images
    def split_images(self, img):
        """Per-view dict of [3,H,W] rgb and [H,W] depth/unc/T/last views into the flat buffers."""
        out = []
        for v, c in enumerate(self.cams):
            p0, P = int(self.pix_base[v]), c.width * c.height
            d = {}
            if img.get("rgb") is not None:
                d["rgb"] = img["rgb"][3 * p0:3 * (p0 + P)].view(3, c.height, c.width)
            for k in ("depth", "unc", "T", "last", "n_contrib"):
                if img.get(k) is not None:
                    d[k] = img[k][p0:p0 + P].view(c.height, c.width)
            out.append(d)
        return out


def render_small(gmap: GaussianMapTensors, cams, params: RenderParams = RenderParams(), images=None,
                 status: Optional[torch.Tensor] = None, stream=None):
    """Forward render of a small map in one launch (gs_render_small): the images of
    Frame.forward bit for bit, without records, bins or workspace.  `cams`: camera objects,
    or their gs_camera records already on the device (then pass `images`).  Returns (images,
    status tensor); after a synchronise, `status & GS_FLAG_PAIR_OVERFLOW` means a tile held
    more than GS_SMALL_MAX_LIST Gaussians and was not written (render with a Frame)."""
    on_device = isinstance(cams, torch.Tensor)   # gs_camera records already on the device (uint8 [80 V])
    n_views = cams.numel() // CAMERA_DTYPE.itemsize if on_device else len(cams)
    if gmap.n > L.GS_SMALL_MAX_GAUSSIANS or n_views > L.GS_SMALL_MAX_VIEWS:
        raise ValueError("render_small takes at most %d Gaussians and %d views" %
                         (L.GS_SMALL_MAX_GAUSSIANS, L.GS_SMALL_MAX_VIEWS))
    if images is None and on_device:
        raise ValueError("pass the images when the cameras are already on the device")
    dev = gmap.mo.device
    cams_dev = cams if on_device else cameras_to_device(cams, dev)
    if images is None:
        P = int(tile_grid(cams, params)[3][-1])
        images = dict(rgb=torch.empty(3 * P, dtype=torch.float32, device=dev),
                      depth=torch.empty(P, dtype=torch.float32, device=dev),
                      unc=torch.empty(P, dtype=torch.float32, device=dev),
                      T=torch.empty(P, dtype=torch.float32, device=dev),
                      last=torch.empty(P, dtype=torch.int32, device=dev), n_contrib=None)
    st = torch.zeros(1, dtype=torch.int32, device=dev) if status is None else status
    _require(st, "status", 1, torch.int32)
    c_img = L.gs_image(_ptr(images.get("rgb")), _ptr(images.get("depth")), _ptr(images.get("unc")),
                       _ptr(images.get("T")), _ptr(images.get("last")), _ptr(images.get("n_contrib")))
    m = gmap.c()
    prm = params.c()
    _timed("gs_render_small", stream, lambda: L.check(
        L.lib().gs_render_small(ctypes.byref(m), _ptr(cams_dev), n_views, ctypes.byref(prm), ctypes.byref(c_img),
                                _ptr(st), _stream(stream)), "gs_render_small"))
    return images, st


class StaleFrameError(RuntimeError):
    """backward() of a render whose Frame has been projected or binned again since its forward."""


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mo, su, q, rgb, frame: Frame):
        gmap = GaussianMapTensors(mo, su, q, rgb)
        img = frame.forward(gmap)
        ctx.frame = frame
        ctx.generation = frame.generation
        ctx.img = img
        ctx.save_for_backward(mo, su, q, rgb)
        # the uncertainty channel has no adjoint (u_i is not a learned parameter, and the
        # backward kernel replays colour and depth only): no gradient flows through it
        ctx.mark_non_differentiable(img["unc"])
        return img["rgb"], img["depth"], img["unc"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_unc):
        if ctx.frame.generation != ctx.generation:
            raise StaleFrameError(
                "the Frame was projected or binned again after this render's forward pass; its records and "
                "tile lists no longer belong to this render.  Give each render that is differentiated together "
                "its own Frame, or call backward before the next render through the same Frame.")
        mo, su, q, rgb = ctx.saved_tensors
        gmap = GaussianMapTensors(mo, su, q, rgb)
        g_rgb = None if g_rgb is None else g_rgb.contiguous()
        g_depth = None if g_depth is None else g_depth.contiguous()
        g = ctx.frame.render_bwd(gmap, ctx.img, g_rgb, g_depth)
        return g["dmo"], g["dsu"], g["dq"], g["drgb"], None


def render(mo, su, q, rgb, frame: Frame):
    """Differentiable render of all views of `frame`: flat (rgb [3P], depth [P], unc [P]) tensors.

    Gradients flow to mo (means, opacity logit), su (log-scales; the uncertainty
    column gets zero), q and rgb through gs_render_bwd, from the rgb and depth
    outputs.  The uncertainty output is marked non-differentiable (the backward pass
    has no adjoint for it).  The backward pass replays the frame's records and tile
    lists: rendering through the same frame again before backward() makes that
    backward() raise StaleFrameError instead of returning wrong gradients.
    """
    return _RenderFn.apply(mo, su, q, rgb, frame)


class InfoGain:
    """Batched information gain over a fixed candidate set (gs_info_gain_batch)."""

    def __init__(self, n: int, cams: Sequence, params: RenderParams = RenderParams(),
                 pair_capacity: Optional[int] = None, device="cuda", record_capacity: Optional[int] = None):
        self.device = torch.device(device)
        self.params = params
        self.c_params = params.c()
        self.cams = list(cams)
        self.V = len(self.cams)
        self.n = int(n)
        self.cams_dev = cameras_to_device(self.cams, self.device)
        _, _, tile_base, _ = tile_grid(self.cams, params)
        self.n_tiles = max(int(tile_base[-1]), 1)
        if pair_capacity is None:
            pair_capacity = min(max(1 << 20, 2 * self.n * self.V), (1 << 31) - 1)
        # records: at most n * V; a smaller capacity (large batches) grows on overflow
        self.record_capacity = int(record_capacity) if record_capacity else self.n * self.V
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.out = torch.zeros(self.V, dtype=torch.float32, device=self.device)
        self._alloc(int(pair_capacity))

    def _alloc(self, pair_capacity):
        self.pair_capacity = pair_capacity
        ws = L.workspace_size(L.GS_OP_INFO_GAIN, self.n, self.V, self.record_capacity, pair_capacity, self.n_tiles)
        self.ws = None
        torch.cuda.empty_cache()
        self.ws = torch.empty(ws, dtype=torch.uint8, device=self.device)

    def __call__(self, gmap: GaussianMapTensors, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        o = self.out if out is None else out
        _require(o, "out", self.V)
        m = gmap.c()
        _timed("gs_info_gain_batch", stream, lambda: L.check(
            L.lib().gs_info_gain_batch(ctypes.byref(m), _ptr(self.cams_dev), self.V, ctypes.byref(self.c_params),
                                       L.GS_IG_RENDER_MEAN, _ptr(o), _ptr(self.status), self.record_capacity,
                                       self.pair_capacity, self.n_tiles, _ptr(self.ws), self.ws.numel(),
                                       _stream(stream)),
            "gs_info_gain_batch"))
        return o

    def read_status(self) -> int:
        flags = ctypes.c_uint32(0)
        L.lib().gs_read_status(_ptr(self.status), ctypes.byref(flags))
        return int(flags.value)

    def grow_if_needed(self) -> bool:
        """After a synchronised call: if records or pairs overflowed, double that capacity (returns True)."""
        f = self.read_status()
        if f & (L.GS_FLAG_PAIR_OVERFLOW | L.GS_FLAG_RECORD_OVERFLOW):
            self.status.zero_()
            if f & L.GS_FLAG_RECORD_OVERFLOW:
                self.record_capacity = min(2 * self.record_capacity, self.n * self.V, (1 << 32) - 2)
            pc = self.pair_capacity
            if f & L.GS_FLAG_PAIR_OVERFLOW:
                pc = min(2 * self.pair_capacity, (1 << 32) - 2)
            self._alloc(pc)
            return True
        return False


# ------------------------------------------------------- render-free view utility (Sec. IV-A/B)
# Values of Sec. IV-C: Gaussian regions of 2.5 m, lambda_xi = 1 (Eq. view_util),
# lambda_g = 3 (the collision test's radius scale, Sec. IV-B)
REGION_SIZE_M = 2.5
LAMBDA_XI = 1.0
LAMBDA_G = 3.0


def uncertainty_update(mo_prev: torch.Tensor, mo_cur: torch.Tensor, su: torch.Tensor, squared: bool = False,
                       stream=None):
    """u = |mu_cur - mu_prev| (or its square) into su[:, 3] for Gaussians whose mean moved
    (gs_uncertainty_update); the others keep their u."""
    for t in (mo_prev, mo_cur, su):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.dim() != 2 or t.shape[1] != 4:
            raise ValueError("expected contiguous float32 CUDA tensors of shape [N, 4]")
    L.check(L.lib().gs_uncertainty_update(_ptr(mo_prev), _ptr(mo_cur), _ptr(su), int(su.shape[0]),
                                          L.GS_U_SQ if squared else L.GS_U_ABS, _stream(stream)),
            "gs_uncertainty_update")


class ViewUtility:
    """Render-free utility xi of candidate poses (Eq. view_util; gs_view_utility_batch).

    thresholds(): mean and sigma of u, high / low thresholds mean +- sigma / 2 (device double[5]);
    __call__: xi per view (mode GS_XI: visible |G_H| - lambda |G_L|; GS_XI_SUM: sum of u over
    the visible Gaussians) and, for GS_XI, the visible counts [V, 2]."""

    def __init__(self, cams: Sequence, near_plane: float = 0.2, range_m: float = 5.0, lam: float = LAMBDA_XI,
                 ground_z: float = float("-inf"), device="cuda"):
        self.device = torch.device(device)
        self.cams = list(cams)
        self.V = len(self.cams)
        self.cams_dev = cameras_to_device(self.cams, self.device)
        self.prm = L.gs_utility_params(near_plane, range_m, lam, ground_z)
        self.stats = torch.zeros(5, dtype=torch.float64, device=self.device)
        self.xi = torch.zeros(self.V, dtype=torch.float32, device=self.device)
        self.counts = torch.zeros((self.V, 2), dtype=torch.int32, device=self.device)
        self.ws_t = torch.empty(max(L.workspace_size(L.GS_OP_THRESHOLDS, 0, 1), 256), dtype=torch.uint8,
                                device=self.device)
        self.ws_u = torch.empty(max(L.workspace_size(L.GS_OP_VIEW_UTILITY, 0, self.V), 256), dtype=torch.uint8,
                                device=self.device)

    def thresholds(self, gmap: GaussianMapTensors, stream=None) -> torch.Tensor:
        m = gmap.c()
        _timed("gs_uncertainty_thresholds", stream, lambda: L.check(
            L.lib().gs_uncertainty_thresholds(ctypes.byref(m), self.prm.ground_z, _ptr(self.stats), _ptr(self.ws_t),
                                              self.ws_t.numel(), _stream(stream)), "gs_uncertainty_thresholds"))
        return self.stats

    def __call__(self, gmap: GaussianMapTensors, mode: int = 0, stats: Optional[torch.Tensor] = None,
                 stream=None):
        m = gmap.c()
        st = self.stats if stats is None else stats
        cnt = self.counts if mode == L.GS_XI else None
        _timed("gs_view_utility_batch", stream, lambda: L.check(
            L.lib().gs_view_utility_batch(ctypes.byref(m), _ptr(self.cams_dev), self.V, ctypes.byref(self.prm), mode,
                                          _ptr(st), _ptr(self.xi), _ptr(cnt), _ptr(self.ws_u), self.ws_u.numel(),
                                          _stream(stream)), "gs_view_utility_batch"))
        return self.xi


def trajectory_utility(vu: "ViewUtility", gmap: GaussianMapTensors, n_traj: int, n_states: int, mode: int = 0,
                       stream=None):
    """Eq. traj_utility over the poses of `vu` (state l of trajectory t at index t * n_states + l):
    (per-trajectory sum of xi [n_traj], index of the best trajectory).  For GS_XI the
    thresholds of vu (vu.thresholds) are used."""
    if n_traj * n_states != vu.V:
        raise ValueError("the ViewUtility must hold n_traj * n_states poses")
    out = torch.zeros(n_traj, dtype=torch.float32, device=vu.device)
    best = torch.zeros(1, dtype=torch.int32, device=vu.device)
    ws = torch.empty(max(L.workspace_size(L.GS_OP_TRAJECTORY, gmap.n, vu.V), 256), dtype=torch.uint8,
                     device=vu.device)
    m = gmap.c()
    L.check(L.lib().gs_trajectory_utility(ctypes.byref(m), _ptr(vu.cams_dev), n_traj, n_states, ctypes.byref(vu.prm),
                                          mode, _ptr(vu.stats), _ptr(out), _ptr(best), _ptr(ws), ws.numel(),
                                          _stream(stream)), "gs_trajectory_utility")
    return out, best


def collision_check(gmap: GaussianMapTensors, points: torch.Tensor, r_robot: float, lambda_g: float = LAMBDA_G,
                    ground_z: float = float("-inf"), stream=None):
    """Smallest margin |p - mu| - (r_robot + lambda_g r) of every test point over all Gaussians
    and whether it collides (gs_collision_check).  points: CUDA float32 [M, 4] (xyz, -)."""
    if points.dtype != torch.float32 or not points.is_cuda or points.dim() != 2 or points.shape[1] != 4:
        raise ValueError("points must be a CUDA float32 tensor of shape [M, 4]")
    pts = points.contiguous()
    M = int(pts.shape[0])
    margin = torch.empty(max(M, 1), dtype=torch.float32, device=pts.device)
    hit = torch.empty(max(M, 1), dtype=torch.int32, device=pts.device)
    m = gmap.c()
    L.check(L.lib().gs_collision_check(ctypes.byref(m), _ptr(pts), M, float(r_robot), float(lambda_g),
                                       float(ground_z), _ptr(margin), _ptr(hit), _stream(stream)),
            "gs_collision_check")
    return margin[:M], hit[:M]


def region_uncertainty(gmap: GaussianMapTensors, origin, size: float, dims, stream=None):
    """Mean u of every cuboid region (gs_region_uncertainty): (omega [R], count [R]),
    region index (iz * dims[1] + iy) * dims[0] + ix.  The paper's regions have size
    REGION_SIZE_M."""
    grid = L.gs_region_grid((ctypes.c_float * 3)(*origin), float(size), (ctypes.c_int32 * 3)(*dims))
    R = int(dims[0]) * int(dims[1]) * int(dims[2])
    dev = gmap.mo.device
    omega = torch.zeros(R, dtype=torch.float32, device=dev)
    count = torch.zeros(R, dtype=torch.int32, device=dev)
    ws = torch.empty(max(L.workspace_size(L.GS_OP_REGIONS, gmap.n, 1, R), 256), dtype=torch.uint8, device=dev)
    m = gmap.c()
    L.check(L.lib().gs_region_uncertainty(ctypes.byref(m), ctypes.byref(grid), _ptr(omega), _ptr(count), _ptr(ws),
                                          ws.numel(), _stream(stream)), "gs_region_uncertainty")
    return omega, count


# ---------------------------------------------------------------------- mapping loss (Eq. 3)
EQ3_WEIGHTS = (1.0, 0.4, 0.1)          # (w_depth, w_rgb = lambda_1, w_ssim = lambda_2), Eq. 3
L1_WEIGHTS = (0.1, 1.0 / 3.0, 0.0)     # mean L1 over RGB elements + 0.1 x mean L1 depth


class ImageLoss:
    """Eq. 3 over the views of a batch (gs_image_loss): loss and dL/d(rgb, depth) in one call.

    sizes: [(width, height)] per view, in the gs_image layout order; weights: (w_depth,
    w_rgb, w_ssim).  __call__ returns (loss4, d_rgb, d_depth), loss4 = device float[4]
    (L, mean |d - d_ref|, mean |c - c_ref|_1, SSIM or NaN when w_ssim = 0); the gradient
    buffers are reused by every call."""

    def __init__(self, sizes, weights=EQ3_WEIGHTS, device="cuda"):
        self.device = torch.device(device)
        self.sizes = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32).reshape(-1, 2))
        self.V = len(self.sizes)
        self.P = int((self.sizes[:, 0].astype(np.int64) * self.sizes[:, 1]).sum())
        self.w = L.gs_loss_weights(*[float(x) for x in weights])
        nb = ctypes.c_size_t(0)
        L.check(L.lib().gs_image_loss_workspace_size(self.sizes.ctypes.data, self.V, ctypes.byref(nb)),
                "gs_image_loss_workspace_size")
        self.ws = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.device)
        self.loss = torch.zeros(4, dtype=torch.float32, device=self.device)
        self.d_rgb = torch.zeros(3 * self.P, dtype=torch.float32, device=self.device)
        self.d_depth = torch.zeros(self.P, dtype=torch.float32, device=self.device)

    @staticmethod
    def for_cameras(cams, weights=EQ3_WEIGHTS, device="cuda") -> "ImageLoss":
        return ImageLoss([(c.width, c.height) for c in cams], weights, device)

    def __call__(self, rgb, depth, rgb_ref, depth_ref, with_grad: bool = True, stream=None):
        for t, n in ((rgb, 3 * self.P), (rgb_ref, 3 * self.P), (depth, self.P), (depth_ref, self.P)):
            if t is not None and (t.numel() != n or t.dtype != torch.float32 or not t.is_contiguous()
                                  or not t.is_cuda):
                raise ValueError("images must be contiguous float32 CUDA tensors in the gs_image layout")
        dr = self.d_rgb if with_grad else None
        dd = self.d_depth if with_grad else None
        _timed("gs_image_loss", stream, lambda: L.check(
            L.lib().gs_image_loss(self.sizes.ctypes.data, self.V, _ptr(rgb), _ptr(depth), _ptr(rgb_ref),
                                  _ptr(depth_ref), ctypes.byref(self.w), _ptr(self.loss), _ptr(dr), _ptr(dd),
                                  _ptr(self.ws), self.ws.numel(), _stream(stream)), "gs_image_loss"))
        return self.loss, dr, dd


class _ImageLossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rgb, depth, rgb_ref, depth_ref, fn: ImageLoss):
        loss, d_rgb, d_depth = fn(rgb.detach(), depth.detach(), rgb_ref, depth_ref)
        ctx.save_for_backward(d_rgb.clone(), d_depth.clone())
        return loss[0].clone()

    @staticmethod
    def backward(ctx, g):
        d_rgb, d_depth = ctx.saved_tensors
        return d_rgb * g, d_depth * g, None, None, None


def image_loss(rgb, depth, rgb_ref, depth_ref, fn: ImageLoss):
    """Differentiable Eq. 3 loss (scalar) of rendered images against references."""
    return _ImageLossFn.apply(rgb, depth, rgb_ref, depth_ref, fn)


# ---------------------------------------------------------------------- optimiser (gs_adam_step)
class Adam:
    """Adam on float32 tensors in place (gs_adam_step): one kernel over all of them, with the
    step count on the device so that the update can be captured in a CUDA graph.  The same
    update as torch.optim.Adam (no weight decay, no amsgrad); tensors need a multiple of 4
    elements and 16-byte alignment.  Gradients are read from each tensor's .grad."""

    def __init__(self, params, lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8):
        self.params = list(params)
        if not 1 <= len(self.params) <= L.GS_ADAM_MAX_TENSORS:
            raise ValueError("between 1 and %d tensors" % L.GS_ADAM_MAX_TENSORS)
        for i, p in enumerate(self.params):
            _require(p, "parameter %d" % i, p.numel())
            if p.numel() % 4:
                raise ValueError("parameter %d: the number of elements must be a multiple of 4" % i)
        dev = self.params[0].device
        with torch.no_grad():
            self.m = [torch.zeros_like(p) for p in self.params]
            self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.prm = L.gs_adam_params(float(lr), float(betas[0]), float(betas[1]), float(eps))
        n = len(self.params)
        self._sizes = (ctypes.c_int64 * n)(*[p.numel() for p in self.params])

    def zero_grad(self, set_to_none: bool = True):
        for p in self.params:
            if set_to_none:
                p.grad = None
            elif p.grad is not None:
                p.grad.zero_()

    def step(self, stream=None):
        n = len(self.params)
        arr = lambda ts: (ctypes.c_void_p * n)(*[_ptr(t) for t in ts])
        grads = [p.grad for p in self.params]
        for i, (p, g) in enumerate(zip(self.params, grads)):
            _require(g, "gradient %d" % i, p.numel())
        _timed("gs_adam_step", stream, lambda: L.check(
            L.lib().gs_adam_step(arr(self.params), arr(grads), arr(self.m), arr(self.v), self._sizes, n,
                                 ctypes.byref(self.prm), _ptr(self.step_count), _stream(stream)), "gs_adam_step"))


# ---------------------------------------------------------------------- tile autotuner
TILE_CANDIDATES = ((16, 16), (16, 8), (8, 8), (32, 8), (32, 16), (32, 32))


def autotune_tiles(gmap: GaussianMapTensors, cams: Sequence, params: RenderParams = RenderParams(),
                   candidates=TILE_CANDIDATES, reps: int = 5, pair_capacity: Optional[int] = None,
                   sweeps: int = 2):
    """Pick a screen tile per resolution class by timing the batched information-gain pass.

    `sweeps` sweeps of coordinate descent over the distinct (width, height) classes of `cams`
    (the second revisits the classes tuned first, with the later classes' new tiles):
    every class starts at the default tile of `params`; in turn, each class's candidates are
    timed on the whole batch with the other classes' current tiles (CUDA events, median of
    `reps` after one warm-up, L2 flushed before each), and the fastest is kept unless the
    class's current tile is within TILE_TUNE_MARGIN of it (a margin on the whole pass, of
    which one class is a part).  Timing the whole batch, not a class
    alone, charges a tile what it costs in the pass that uses it (a class timed alone once
    preferred 8x8 tiles at 160x120 that made the full pass 4% slower).  Returns
    ({(W, H): (tile_w, tile_h)}, {(W, H): {tile: ms}}).  Use `with_tiles` to apply the choice
    to a camera list (the timings are those of the last sweep).
    """
    classes = []
    for c in cams:
        if (c.width, c.height) not in classes:
            classes.append((c.width, c.height))
    choice = {res: (params.tile_w, params.tile_h) for res in classes}
    timings = {res: {} for res in classes}

    def batch_ms(ch) -> float:
        ig = InfoGain(gmap.n, with_tiles(cams, ch), params, pair_capacity=pair_capacity)
        ig(gmap)
        torch.cuda.synchronize()
        while ig.grow_if_needed():
            ig(gmap)
            torch.cuda.synchronize()
        ms = _best_ms(lambda: ig(gmap), reps)
        del ig
        return ms

    for _ in range(max(int(sweeps), 1)):
        for res in classes:
            timings[res] = {}
            for tw, th in candidates:
                if not valid_tile(tw, th):
                    continue
                ch = dict(choice)
                ch[res] = (tw, th)
                timings[res][(tw, th)] = batch_ms(ch)
            choice[res] = _pick(timings[res], choice[res], TILE_TUNE_MARGIN)
    return choice, timings


IG_BATCH_CANDIDATES = (4, 8, 16)     # RenderParams.ig_batch
FWD_BATCH_CANDIDATES = (1, 2, 4)     # RenderParams.fwd_batch


L2_FLUSH_BYTES = 256 << 20     # more than the GPU's L2: written between timed calls of the autotuners
TUNE_MARGIN = 0.03             # a candidate replaces the default only if it is faster by more than this
# ... of the whole batch when one class's tile changes: that class is only part of the pass
TILE_TUNE_MARGIN = 0.01


def _best_ms(fn, reps: int) -> float:
    """Median device time of `fn` over `reps` calls (CUDA events on the current stream), after
    one warm-up, with the L2 cache flushed before every timed call (as the steps it tunes run).
    The median, not the minimum: a single fast outlier must not decide a choice."""
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    fn()
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    del flush
    return float(np.median(t))


def _pick(timings, default, margin: float = TUNE_MARGIN):
    """The fastest key, unless the default (when timed) is within `margin` of it."""
    best = min(timings, key=timings.get)
    if default in timings and timings[default] <= timings[best] * (1.0 + margin):
        return default
    return best


def autotune_ig_batch(gmap: GaussianMapTensors, cams: Sequence, params: RenderParams = RenderParams(),
                      candidates=IG_BATCH_CANDIDATES, reps: int = 7, pair_capacity: Optional[int] = None):
    """Pick the chunk depth of the information-gain compositing (RenderParams.ig_batch) by timing
    the batched pass over `cams` (with their own tiles, e.g. from autotune_tiles) at each
    candidate; the scores are the same for every depth.  Returns (depth, {depth: ms})."""
    from dataclasses import replace
    timings = {}
    for b in candidates:
        ig = InfoGain(gmap.n, cams, replace(params, ig_batch=int(b)), pair_capacity=pair_capacity)
        ig(gmap)
        torch.cuda.synchronize()
        while ig.grow_if_needed():
            ig(gmap)
            torch.cuda.synchronize()
        timings[int(b)] = _best_ms(lambda: ig(gmap), reps)
        del ig
    torch.cuda.empty_cache()
    return _pick(timings, 8), timings


def autotune_mapping(gmap: GaussianMapTensors, cams: Sequence, params: RenderParams = RenderParams(),
                     tiles=TILE_CANDIDATES, batches=FWD_BATCH_CANDIDATES, reps: int = 7):
    """Pick the keyframes' tile (RenderParams.tile_w, tile_h) and the forward chunk depth
    (RenderParams.fwd_batch) of a mapping step by timing one forward and backward pass of the
    map through all `cams` (unit image gradients): the tile first at the default depth, then
    the depth at that tile.  Returns (params, {(tile_w, tile_h, fwd_batch): ms})."""
    from dataclasses import replace
    timings = {}

    def time_step(prm):
        fr = Frame(gmap.n, cams, prm, with_pair_tiles=False)
        img = fr.forward(gmap)
        torch.cuda.synchronize()
        while fr.grow_if_needed():
            img = fr.forward(gmap)
            torch.cuda.synchronize()
        d_rgb, d_dep = torch.ones_like(img["rgb"]), torch.ones_like(img["depth"])
        grads = {k: torch.empty((gmap.n, 4), dtype=torch.float32, device=fr.device) for k in ("dmo", "dsu", "dq", "drgb")}

        def step():
            fr.forward(gmap, img)
            fr.render_bwd(gmap, img, d_rgb, d_dep, grads)

        ms = _best_ms(step, reps)
        del fr, img, grads
        return ms

    d_batch = params.fwd_batch or 2
    for tw, th in tiles:
        if not valid_tile(tw, th):
            continue
        prm = replace(params, tile_w=int(tw), tile_h=int(th), fwd_batch=d_batch)
        timings[(int(tw), int(th), d_batch)] = time_step(prm)
    tw, th, _ = _pick(timings, (params.tile_w, params.tile_h, d_batch))
    for b in batches:
        prm = replace(params, tile_w=tw, tile_h=th, fwd_batch=int(b))
        key = (tw, th, int(b))
        if key not in timings:
            timings[key] = time_step(prm)
    best = _pick({k: v for k, v in timings.items() if k[:2] == (tw, th)}, (tw, th, d_batch))
    torch.cuda.empty_cache()
    return replace(params, tile_w=best[0], tile_h=best[1], fwd_batch=best[2]), timings


def with_tiles(cams: Sequence, choice) -> list:
    """Cameras with their tile size set from an autotune_tiles choice ({(W, H): (tile_w, tile_h)})."""
    out = []
    for c in cams:
        tw, th = choice.get((c.width, c.height), (0, 0))
        out.append(type(c)(c.fx, c.fy, c.cx, c.cy, c.width, c.height, c.R, c.T, tw, th))
    return out
