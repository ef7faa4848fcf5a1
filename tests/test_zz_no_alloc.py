"""gs_render_bwd_noalloc: the backward pass for callers that cannot allocate.

Such callers (a real-time loop that reserved all its device memory at start-up,
a plugin that only gets its host's buffers, code inside someone else's graph
capture) cannot hand gs_render_bwd a workspace; this entry point keeps the
scratch in a fixed array of the library instead.  Its results must equal the
workspace version's on the same inputs, on consecutive calls (the shared
array keeps the previous call's contents, which must not leak into the next).

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_18122_gb300 import _lib as L
from paper_2409_18122_gb300 import gs, scenes

from gpu_helpers import compare_grads

pytestmark = pytest.mark.gpu


def _call_noalloc(fr, gm, img, d_rgb, d_dep, out):
    c_img = L.gs_image(*(ctypes.c_void_p(t.data_ptr()) if t is not None else None
                         for t in (img["rgb"], img["depth"], img["unc"], img["T"], img["last"])), None)
    c_g = L.gs_image_grad(ctypes.c_void_p(d_rgb.data_ptr()), ctypes.c_void_p(d_dep.data_ptr()))
    c_out = L.gs_map_grad(*(ctypes.c_void_p(out[k].data_ptr()) for k in ("dmo", "dsu", "dq", "drgb")))
    m = gm.c()
    return L.lib().gs_render_bwd_noalloc(ctypes.byref(m), ctypes.byref(fr.c_proj), ctypes.byref(fr.c_bins),
                                         ctypes.byref(c_img), ctypes.byref(c_g), ctypes.c_void_p(fr.cams_dev.data_ptr()),
                                         fr.V, ctypes.byref(fr.c_params), ctypes.byref(c_out),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_backward_matches_workspace_backward_twice():
    sc = scenes.config0()
    gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
    fr = gs.Frame(gm.n, sc.cams)
    assert fr.rec_capacity <= L.GS_NOALLOC_MAX_RECORDS
    img = fr.forward(gm)
    rng = np.random.default_rng(4)
    for call in range(2):
        d_rgb = torch.from_numpy(rng.normal(size=img["rgb"].numel()).astype(np.float32)).cuda()
        d_dep = torch.from_numpy(rng.normal(size=img["depth"].numel()).astype(np.float32)).cuda()
        ref = fr.render_bwd(gm, img, d_rgb, d_dep)
        out = {k: torch.full((gm.n, 4), float("nan"), device="cuda") for k in ("dmo", "dsu", "dq", "drgb")}
        assert _call_noalloc(fr, gm, img, d_rgb, d_dep, out) == L.GS_OK
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        want = {k: v.cpu().numpy().astype(np.float64) for k, v in ref.items()}
        assert all(np.isfinite(v).all() for v in got.values())
        compare_grads(got, want, what="noalloc call %d" % call)


def test_noalloc_rejects_records_beyond_its_scratch():
    sc = scenes.config0()
    gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
    fr = gs.Frame(gm.n, sc.cams)
    img = fr.forward(gm)
    big = L.gs_proj(*[getattr(fr.c_proj, f) for f, _ in L.gs_proj._fields_])
    big.capacity = L.GS_NOALLOC_MAX_RECORDS + 1
    d = torch.zeros(img["rgb"].numel(), device="cuda")
    out = {k: torch.zeros((gm.n, 4), device="cuda") for k in ("dmo", "dsu", "dq", "drgb")}
    c_img = L.gs_image(*(ctypes.c_void_p(img[k].data_ptr()) for k in ("rgb", "depth", "unc", "T", "last")), None)
    c_g = L.gs_image_grad(ctypes.c_void_p(d.data_ptr()), None)
    c_out = L.gs_map_grad(*(ctypes.c_void_p(out[k].data_ptr()) for k in ("dmo", "dsu", "dq", "drgb")))
    m = gm.c()
    st = L.lib().gs_render_bwd_noalloc(ctypes.byref(m), ctypes.byref(big), ctypes.byref(fr.c_bins), ctypes.byref(c_img),
                                       ctypes.byref(c_g), ctypes.c_void_p(fr.cams_dev.data_ptr()), fr.V,
                                       ctypes.byref(fr.c_params), ctypes.byref(c_out), None)
    assert st == L.GS_ERR_WORKSPACE


def test_noalloc_checks_its_arguments_like_the_workspace_backward():
    """The arguments gs_render_bwd refuses are refused here too, with the same codes, before
    anything is enqueued: a tile capacity past 2^27 - 1, no views or too many, bad rendering
    constants, a misaligned camera array."""
    sc = scenes.config0()
    gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
    fr = gs.Frame(gm.n, sc.cams)
    img = fr.forward(gm)
    torch.cuda.synchronize()
    d = torch.zeros(img["rgb"].numel(), device="cuda")
    out = {k: torch.zeros((gm.n, 4), device="cuda") for k in ("dmo", "dsu", "dq", "drgb")}
    c_img = L.gs_image(*(ctypes.c_void_p(img[k].data_ptr()) for k in ("rgb", "depth", "unc", "T", "last")), None)
    c_g = L.gs_image_grad(ctypes.c_void_p(d.data_ptr()), None)
    c_out = L.gs_map_grad(*(ctypes.c_void_p(out[k].data_ptr()) for k in ("dmo", "dsu", "dq", "drgb")))
    m = gm.c()
    cams = ctypes.c_void_p(fr.cams_dev.data_ptr())

    def both(bins=fr.c_bins, n_views=fr.V, prm=fr.c_params, cam=cams):
        a = L.lib().gs_render_bwd_noalloc(ctypes.byref(m), ctypes.byref(fr.c_proj), ctypes.byref(bins),
                                          ctypes.byref(c_img), ctypes.byref(c_g), cam, n_views, ctypes.byref(prm),
                                          ctypes.byref(c_out), None)
        b = L.lib().gs_render_bwd(ctypes.byref(m), ctypes.byref(fr.c_proj), ctypes.byref(bins), ctypes.byref(c_img),
                                  ctypes.byref(c_g), cam, n_views, ctypes.byref(prm), ctypes.byref(c_out),
                                  ctypes.c_void_p(fr.ws.data_ptr()), fr.ws.numel(), None)
        return a, b

    big_tiles = L.gs_bins(*[getattr(fr.c_bins, f) for f, _ in L.gs_bins._fields_])
    big_tiles.tile_capacity = 1 << 27
    assert both(bins=big_tiles) == (L.GS_ERR_ARG, L.GS_ERR_ARG)
    assert both(n_views=0) == (L.GS_ERR_ARG, L.GS_ERR_ARG)
    assert both(n_views=(1 << 20) + 1) == (L.GS_ERR_ARG, L.GS_ERR_ARG)
    for field, bad in (("T_min", 1.5), ("eps2d", -1.0), ("near_plane", 0.0), ("guard", 0.0)):
        prm = L.gs_params(*[getattr(fr.c_params, f) for f, _ in L.gs_params._fields_])
        setattr(prm, field, bad)
        assert both(prm=prm) == (L.GS_ERR_ARG, L.GS_ERR_ARG), field
    assert both(cam=ctypes.c_void_p(fr.cams_dev.data_ptr() + 2)) == (L.GS_ERR_ALIGN, L.GS_ERR_ALIGN)
    torch.cuda.synchronize()
    assert all(float(t.abs().max()) == 0.0 for t in out.values())   # nothing ran
