"""Failure paths of the CUDA path, made on the host: bad map entries and bad cameras are
written into the inputs before the call, and the tests check the device status word and
that the valid part of the output still equals the oracle's.  Nothing here is expected to
fault: every bad value is one the library's own checks turn into a status flag.

Sec. III of RT-GuIDE (projection and compositing) and Eq. (nbv) (information gain); the
tolerances are those of gpu_helpers.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2409_18122_gb300 import gs, scenes
from paper_2409_18122_gb300 import _lib as L
from paper_2409_18122_gb300.scenes import Camera

from gpu_helpers import IG_RTOL, compare_image, gpu_records, images_host

pytestmark = pytest.mark.gpu

SENTINEL = -7.0


def _visible_ids(gmap, cams, k, seed):
    vis = O.project(gmap, cams)["vis"].any(axis=0)
    ids = np.nonzero(vis)[0]
    return np.random.default_rng(seed).choice(ids, size=k, replace=False)


def test_nonfinite_parameters_are_culled_like_removed_gaussians():
    """NaN or Inf in the mean, the opacity logit, a log-scale or the quaternion of some visible
    Gaussians: GS_FLAG_NONFINITE is set (informational, not an error), those Gaussians get no
    record, and images and information gain equal the oracle's for the map without them."""
    sc = scenes.config0()
    cams = sc.cams + [Camera(90, 90, 40, 30, 80, 60)]
    g = sc.gmap.copy()
    bad = _visible_ids(g, cams, 8, 5)
    g.mo[bad[0], 0] = np.nan
    g.mo[bad[1], 2] = np.inf
    g.mo[bad[2], 3] = np.nan            # opacity logit
    g.mo[bad[3], 3] = -np.inf
    g.su[bad[4], 1] = np.inf            # log-scale
    g.su[bad[5], 0] = np.nan
    g.q[bad[6], 2] = np.nan             # quaternion
    g.q[bad[7], 0] = -np.inf
    keep = np.setdiff1d(np.arange(g.n), bad)
    clean = sc.gmap.subset(keep)
    gm = gs.GaussianMapTensors.from_numpy(g)
    fr = gs.Frame(gm.n, cams)
    img = fr.forward(gm)
    torch.cuda.synchronize()
    flags = fr.read_status()
    assert flags & L.GS_FLAG_NONFINITE and not flags & L.GS_FLAG_ERROR_MASK
    rec = gpu_records(fr)
    assert not np.isin(rec["gid"], bad).any()
    ref = O.render_images(clean, cams)
    for v, h in enumerate(images_host(fr, img)):
        compare_image(h, ref[v], "view %d" % v)
    ig_op = gs.InfoGain(gm.n, cams)
    ig = ig_op(gm).cpu().numpy().astype(np.float64)
    assert ig_op.read_status() & L.GS_FLAG_NONFINITE
    ref_ig = np.array([im["unc"].mean() for im in ref])
    np.testing.assert_allclose(ig, ref_ig, rtol=IG_RTOL, atol=1e-7)


def _bad_camera_batch():
    sc = scenes.config0()
    good0, good1 = sc.cams[0], Camera(90, 90, 40, 30, 80, 60)
    cams = [good0,
            Camera(-100.0, 100.0, 64.0, 48.0, 128, 96),             # fx <= 0
            Camera(100.0, 100.0, 0.0, 48.0, 0, 96),                 # W = 0
            good1,
            Camera(100.0, 100.0, 32.0, 24.0, 64, 48).with_tile(12, 8),   # invalid per-view tile
            Camera(100.0, 0.0, 32.0, 24.0, 64, 48)]                 # fy = 0
    return sc.gmap, cams, [0, 3]


def test_bad_cameras_are_flagged_and_leave_the_valid_views_intact():
    """Cameras with fx <= 0, fy = 0, W = 0 and an invalid tile among valid ones: GS_FLAG_BAD_CAMERA
    is set, the bad views get no records, tiles or pixel writes (their image region keeps what
    the caller put there), and the valid views equal the oracle's."""
    gmap, cams, good = _bad_camera_batch()
    assert [gs.camera_ok(c, gs.RenderParams()) for c in cams] == [v in good for v in range(len(cams))]
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    fr = gs.Frame(gm.n, cams)
    img = fr.new_images(with_counts=True)
    for t in img.values():
        t.fill_(SENTINEL if t.dtype == torch.float32 else -7)
    fr.forward(gm, img)
    torch.cuda.synchronize()
    assert fr.read_status() & L.GS_FLAG_BAD_CAMERA
    assert set(np.unique(gpu_records(fr)["view"]).tolist()) <= set(good)
    views = images_host(fr, img)
    ref = O.render_images(gmap, [cams[v] for v in good])
    for k, v in enumerate(good):
        compare_image(views[v], ref[k], "view %d" % v)
    for v, c in enumerate(cams):
        if v in good:
            continue
        h = views[v]
        assert h["T"].size == max(c.width, 0) * max(c.height, 0)
        for key in ("rgb", "depth", "unc", "T"):
            assert (h[key] == SENTINEL).all(), (v, key)
        assert (h["last"] == -7).all()
    # the whole buffer holds exactly the views' pixels: nothing past the last view
    assert img["T"].numel() == sum(max(c.width, 0) * max(c.height, 0) for c in cams)


def test_bad_cameras_in_an_information_gain_batch():
    """The same batch scored by gs_info_gain_batch: the flag is set, the bad views score 0 and
    the valid ones equal the oracle's and their own single-view calls."""
    gmap, cams, good = _bad_camera_batch()
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    ig_op = gs.InfoGain(gm.n, cams)
    ig = ig_op(gm).cpu().numpy()
    assert ig_op.read_status() & L.GS_FLAG_BAD_CAMERA
    ref, _ = O.info_gain(gmap, [cams[v] for v in good])
    for k, v in enumerate(good):
        assert abs(float(ig[v]) - ref[k]) <= IG_RTOL * abs(ref[k]) + 1e-7, (v, ig[v], ref[k])
        assert gs.InfoGain(gm.n, [cams[v]])(gm).cpu().numpy()[0] == ig[v]
    for v in range(len(cams)):
        if v not in good:
            assert ig[v] == 0.0, (v, ig[v])
