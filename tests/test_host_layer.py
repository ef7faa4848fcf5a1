"""Host-side logic of the Python layer, on the CPU: camera records, the tile grid, tile
choices, the per-view image views and the capacity growth after an overflow.  Buffers are
allocated on the CPU device (the layer computes sizes and pointers only; no kernel runs)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2409_18122_gb300 import _lib as L
from paper_2409_18122_gb300 import gs
from paper_2409_18122_gb300.scenes import Camera


def _cams():
    return [Camera(100, 100, 60, 40, 120, 80), Camera(50, 50, 20, 15, 40, 30).with_tile(8, 8),
            Camera(80, 80, 16.5, 9.5, 33, 19).with_tile(32, 8), Camera(10, 10, 0.5, 0.5, 1, 1)]


def test_camera_records_match_the_c_struct():
    """The numpy record the layer uploads has the offsets of gs_camera (checked against the
    header by the ABI test) and carries each camera's own tile size."""
    for name, _ in L.gs_camera._fields_:
        assert gs.CAMERA_DTYPE.fields[name][1] == getattr(L.gs_camera, name).offset, name
    assert gs.CAMERA_DTYPE.itemsize == L.ctypes.sizeof(L.gs_camera)
    cams = _cams()
    a = gs.pack_cameras(cams)
    R = np.arange(9, dtype=np.float32).reshape(3, 3)
    c = Camera(1.5, 2.5, 3.5, 4.5, 7, 9, R=R, T=np.array([1.0, -2.0, 3.0]))
    b = gs.pack_cameras([c])[0]
    assert (b["fx"], b["fy"], b["cx"], b["cy"], b["width"], b["height"]) == (1.5, 2.5, 3.5, 4.5, 7, 9)
    np.testing.assert_array_equal(b["R"], R.reshape(9))
    np.testing.assert_array_equal(b["T"], [1.0, -2.0, 3.0])
    assert [(r["tile_w"], r["tile_h"]) for r in a] == [(0, 0), (8, 8), (32, 8), (0, 0)]
    dev = gs.cameras_to_device(cams, "cpu")
    assert dev.dtype == torch.uint8 and dev.numel() == 80 * len(cams)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_tile_grid_matches_the_oracle(tile):
    """The layer's tile grid (used to size buffers and split images) equals the oracle's,
    per-view tiles included, and its pixel offsets are the running sums of W x H."""
    cams = _cams()
    p = gs.RenderParams(tile_w=tile[0], tile_h=tile[1])
    tx, ty, tile_base, pix_base = gs.tile_grid(cams, p)
    otx, obase = O.tile_grid(cams, O.Params(tile_w=tile[0], tile_h=tile[1]))
    np.testing.assert_array_equal(tx, otx)
    np.testing.assert_array_equal(tile_base, obase)
    np.testing.assert_array_equal(pix_base, np.concatenate([[0], np.cumsum([c.width * c.height for c in cams])]))
    # the 8x8 view of 40x30 has 5 x 4 tiles, the 1x1 view one tile of the default size
    assert (tx[1], ty[1]) == (5, 4) and (tx[3], ty[3]) == (1, 1)


def test_with_tiles_applies_a_choice_per_resolution_class():
    cams = [Camera(50, 50, 40, 30, 80, 60), Camera(90, 90, 80, 60, 160, 120), Camera(50, 50, 40, 30, 80, 60)]
    out = gs.with_tiles(cams, {(80, 60): (8, 8), (160, 120): (16, 8)})
    assert [(c.tile_w, c.tile_h) for c in out] == [(8, 8), (16, 8), (8, 8)]
    assert [(c.width, c.height, c.fx) for c in out] == [(c.width, c.height, c.fx) for c in cams]
    none = gs.with_tiles(cams, {})
    assert all((c.tile_w, c.tile_h) == (0, 0) for c in none)     # 0 = the renderer's default


def test_split_images_views_the_flat_buffers():
    cams = _cams()
    fr = gs.Frame(100, cams, device="cpu")
    P = fr.n_pixels
    img = {"rgb": torch.arange(3 * P, dtype=torch.float32), "T": torch.arange(P, dtype=torch.float32),
           "last": torch.arange(P, dtype=torch.int32)}
    parts = fr.split_images(img)
    assert len(parts) == len(cams)
    p0 = 0
    for c, d in zip(cams, parts):
        n = c.width * c.height
        assert d["rgb"].shape == (3, c.height, c.width) and d["T"].shape == (c.height, c.width)
        # planar per view: channel k of this view starts at 3 p0 + k n
        for k in range(3):
            assert float(d["rgb"][k, 0, 0]) == 3 * p0 + k * n
        assert float(d["T"][-1, -1]) == p0 + n - 1 and int(d["last"][0, 0]) == p0
        assert "depth" not in d
        p0 += n
    assert p0 == P


def _frame_with_status(flags, monkeypatch, n=1000):
    fr = gs.Frame(n, _cams(), device="cpu", record_capacity=64, pair_capacity=4096)
    monkeypatch.setattr(fr, "read_status", lambda: flags)
    return fr


def test_record_overflow_grows_the_record_capacity(monkeypatch):
    """After GS_FLAG_RECORD_OVERFLOW the record buffers are sized for the records the
    projection counted (grp_base[V G], with a margin), never beyond N x V."""
    fr = _frame_with_status(L.GS_FLAG_RECORD_OVERFLOW, monkeypatch)
    fr.grp_base[fr.n_slots] = 500
    assert fr.grow_if_needed()
    assert fr.rec_capacity == int(500 * 1.25) + 1024
    assert fr.splat.shape[0] == fr.rec_capacity and fr.c_proj.capacity == fr.rec_capacity
    assert fr.pair_capacity == 4096
    fr2 = _frame_with_status(L.GS_FLAG_RECORD_OVERFLOW, monkeypatch, n=100)
    fr2.grp_base[fr2.n_slots] = 390
    assert fr2.grow_if_needed() and fr2.rec_capacity == 100 * len(_cams())


def test_pair_overflow_grows_the_pair_capacity(monkeypatch):
    fr = _frame_with_status(L.GS_FLAG_PAIR_OVERFLOW, monkeypatch)
    fr.pair_count[0] = 10_000
    assert fr.grow_if_needed()
    assert fr.pair_capacity == int(10_000 * 1.25) + 1024
    assert fr.pair_rec.numel() == fr.pair_capacity and fr.c_bins.pair_capacity == fr.pair_capacity
    # a saturated count (more pairs than 32 bits hold) doubles the capacity instead
    fr = _frame_with_status(L.GS_FLAG_PAIR_OVERFLOW, monkeypatch)
    fr.pair_count[0] = -1
    assert fr.grow_if_needed() and fr.pair_capacity == int(2 * 4096 * 1.25) + 1024


def test_no_overflow_keeps_the_buffers(monkeypatch):
    fr = _frame_with_status(0, monkeypatch)
    rec, pairs = fr.rec_capacity, fr.pair_capacity
    assert not fr.grow_if_needed()
    assert (fr.rec_capacity, fr.pair_capacity) == (rec, pairs)


def test_workspace_covers_every_stage():
    """The frame's workspace is at least what gs_workspace_size asks for each stage."""
    cams = _cams()
    fr = gs.Frame(5000, cams, device="cpu")
    need = [L.workspace_size(L.GS_OP_PROJECT, fr.n, fr.V),
            L.workspace_size(L.GS_OP_BIN_SORT, fr.n, fr.V, fr.rec_capacity, fr.pair_capacity, fr.n_tiles),
            L.workspace_size(L.GS_OP_RENDER_BWD, fr.n, fr.V, fr.rec_capacity)]
    assert fr.ws.numel() >= max(need)
    ig = gs.InfoGain(5000, cams, device="cpu")
    assert ig.ws.numel() >= L.workspace_size(L.GS_OP_INFO_GAIN, 5000, len(cams), ig.record_capacity,
                                             ig.pair_capacity, ig.n_tiles)


def test_info_gain_growth_doubles_the_overflowed_capacity(monkeypatch):
    """The batched pass has no count to read back cheaply: an overflowed record or pair
    capacity is doubled (records never beyond N x V) and the status word cleared."""
    cams = _cams()
    ig = gs.InfoGain(1000, cams, device="cpu", record_capacity=300, pair_capacity=5000)
    ig.status[0] = 7
    monkeypatch.setattr(ig, "read_status", lambda: L.GS_FLAG_RECORD_OVERFLOW | L.GS_FLAG_PAIR_OVERFLOW)
    assert ig.grow_if_needed()
    assert (ig.record_capacity, ig.pair_capacity) == (600, 10_000) and int(ig.status[0]) == 0
    ig.record_capacity = 3000
    assert ig.grow_if_needed() and ig.record_capacity == 1000 * len(cams)
    monkeypatch.setattr(ig, "read_status", lambda: 0)
    assert not ig.grow_if_needed()


def test_host_tensors_are_refused_before_the_library():
    """Every entry point of the layer checks, before a pointer crosses the C ABI, that the
    tensors it passes are contiguous CUDA tensors of the right type and size (the kernels
    would otherwise be handed host addresses)."""
    cams = _cams()
    fr = gs.Frame(100, cams, device="cpu")
    P = fr.n_pixels
    img = {"rgb": torch.zeros(3 * P), "depth": torch.zeros(P), "unc": None, "T": torch.ones(P),
           "last": torch.zeros(P, dtype=torch.int32)}
    with pytest.raises(ValueError, match="image"):
        fr.render_fwd(None, img)
    with pytest.raises(ValueError, match="image"):
        fr.render_bwd(None, img, torch.zeros(3 * P), torch.zeros(P))
    with pytest.raises(ValueError, match="out"):
        fr.info_gain(torch.zeros(len(cams)))
    ig = gs.InfoGain(100, cams, device="cpu")
    with pytest.raises(ValueError, match="out"):
        ig(None, out=torch.zeros(len(cams)))
    with pytest.raises(ValueError, match="parameter 0"):
        gs.Adam([torch.zeros(8, 4)])
    loss = gs.ImageLoss([(c.width, c.height) for c in cams], device="cpu")
    with pytest.raises(ValueError, match="CUDA"):
        loss(torch.zeros(3 * P), torch.zeros(P), torch.zeros(3 * P), torch.zeros(P))


def test_require_accepts_none_and_checks_type_and_size():
    gs._require(None, "x", 10)
    with pytest.raises(ValueError, match="at least 10"):
        gs._require(torch.zeros(20), "x", 10)          # a host tensor, whatever its size
    with pytest.raises(ValueError):
        gs._require(np.zeros(20, np.float32), "x", 10)  # not a tensor at all


class _FakeFrame:
    """Stands in for gs.Frame on the CPU: forward() bumps the generation like project() and
    bin_sort() do and returns images; render_bwd() returns gradients of ones."""

    def __init__(self, n, P):
        self.n, self.P, self.generation, self.bwd_calls = n, P, 0, 0

    def forward(self, gmap):
        self.generation += 2
        z = torch.zeros(self.P)
        return dict(rgb=torch.zeros(3 * self.P), depth=z.clone(), unc=z.clone(), T=z.clone(),
                    last=torch.zeros(self.P, dtype=torch.int32))

    def render_bwd(self, gmap, img, d_rgb, d_depth):
        self.bwd_calls += 1
        return {k: torch.ones(self.n, 4) for k in ("dmo", "dsu", "dq", "drgb")}


def _params(n=5):
    return [torch.zeros(n, 4, requires_grad=True) for _ in range(4)]


def test_backward_after_a_second_render_through_the_frame_raises():
    """Two renders through one frame, then backward of the first: the records and tile lists it
    would replay belong to the second render, so it raises instead of returning wrong gradients."""
    fr = _FakeFrame(5, 12)
    p = _params()
    rgb1, _, _ = gs.render(*p, fr)
    rgb2, _, _ = gs.render(*p, fr)
    with pytest.raises(gs.StaleFrameError):
        rgb1.sum().backward()
    assert fr.bwd_calls == 0
    rgb2.sum().backward()            # the latest render is still differentiable
    assert fr.bwd_calls == 1 and torch.equal(p[0].grad, torch.ones(5, 4))


def test_uncertainty_output_is_not_differentiable():
    fr = _FakeFrame(5, 12)
    rgb, depth, unc = gs.render(*_params(), fr)
    assert rgb.requires_grad and depth.requires_grad and not unc.requires_grad
    with pytest.raises(RuntimeError):
        unc.sum().backward()


def test_autotuner_keeps_the_default_within_the_margin():
    """A candidate replaces the default only if it is faster by more than TUNE_MARGIN."""
    m = gs.TUNE_MARGIN
    assert gs._pick({"d": 1.0, "a": 1.0 / (1 + m / 2)}, "d") == "d"
    assert gs._pick({"d": 1.0, "a": 1.0 / (1 + 2 * m)}, "d") == "a"
    assert gs._pick({"a": 2.0, "b": 1.0}, "missing") == "b"
    # the tile tuner times whole batches, where one class's change is a part: a smaller margin
    t = gs.TILE_TUNE_MARGIN
    assert t < m
    assert gs._pick({"d": 1.0, "a": 1.0 / (1 + 2 * t)}, "d", t) == "a"
    assert gs._pick({"d": 1.0, "a": 1.0 / (1 + t / 2)}, "d", t) == "d"


def test_tile_and_camera_checks_mirror_the_library():
    """The Python layer's tile and camera checks, which size the buffers, accept exactly what
    the library's do (include/gs.h gs_params, GS_FLAG_BAD_CAMERA)."""
    ok = {(w, h) for w in (8, 16, 32, 64) for h in range(8, 129, 8) if w * h in (64, 128, 256, 512, 1024)}
    for w in range(0, 70):
        for h in range(0, 140):
            assert gs.valid_tile(w, h) == ((w, h) in ok), (w, h)
    p = gs.RenderParams()
    assert gs.camera_ok(Camera(100, 100, 60, 40, 120, 80), p)
    assert not gs.camera_ok(Camera(-100, 100, 60, 40, 120, 80), p)
    assert not gs.camera_ok(Camera(100, 0, 60, 40, 120, 80), p)
    assert not gs.camera_ok(Camera(100, 100, 60, 40, 0, 80), p)
    assert not gs.camera_ok(Camera(100, 100, 60, 40, 120, 80).with_tile(12, 8), p)
    assert not gs.camera_ok(Camera(float("inf"), 100, 60, 40, 120, 80), p)


def test_invalid_cameras_keep_their_pixels_and_lose_their_tiles():
    cams = [Camera(100, 100, 60, 40, 120, 80), Camera(-100, 100, 60, 40, 64, 48),
            Camera(100, 100, 60, 40, 0, 48), Camera(50, 50, 20, 15, 40, 30).with_tile(12, 8)]
    tx, ty, tile_base, pix_base = gs.tile_grid(cams, gs.RenderParams())
    assert list(tx * ty) == [8 * 5, 0, 0, 0]
    assert list(np.diff(pix_base)) == [120 * 80, 64 * 48, 0, 40 * 30]
    assert tile_base[-1] == 40
