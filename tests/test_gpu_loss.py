"""Eq. 3 mapping loss (gs_image_loss) through the C ABI vs the FP64 oracle.

Tolerances come from the FP32 arithmetic of the kernel.  Per pixel, the SSIM moments are
11x11 window sums (relative rounding ~1e-6).  The variances E[x^2] - mu^2 cancel, with an
absolute error ~1e-7 against C2 = 9e-4.  So S carries ~1e-4 relative error at worst in flat
regions and far less on average; the loss is a mean of S, so its error averages down, and
rtol 2e-5 is used for L and its terms.  The SSIM gradient combines blurred derivative planes
of size up to ~1/C2 whose sum is O(1), so its elementwise error is bounded against the
largest SSIM gradient of the view: |g - g_ref| <= 1e-3 max|g_ssim,ref| + 1e-6 |g_ref|.  The
L1 gradient is w sign(dx) / N_p: exact sign (the FP32 difference of FP32 inputs has the
exact sign), so without SSIM the gradient agrees to FP32 rounding of w / N_p."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2409_18122_gb300 import gs

pytestmark = pytest.mark.gpu


def _views(sizes, seed, smooth=True):
    """Render-like images (smooth fields plus noise) and references, in gs_image order."""
    rng = np.random.default_rng(seed)
    rgbs, deps, rrefs, drefs = [], [], [], []
    for (W, H) in sizes:
        yy, xx = np.mgrid[0:H, 0:W] / max(W, H)
        base = 0.5 + 0.3 * np.sin(6 * xx[None] + rng.uniform(0, 6, (3, 1, 1))) * np.cos(4 * yy[None]) if smooth \
            else rng.uniform(0, 1, (3, H, W))
        x = np.clip(base + rng.normal(0, 0.05, (3, H, W)), 0, 1).astype(np.float32)
        y = np.clip(base + rng.normal(0, 0.05, (3, H, W)), 0, 1).astype(np.float32)
        d = (2 + np.sin(3 * xx) + rng.normal(0, 0.02, (H, W))).astype(np.float32)
        dr = (d + rng.normal(0, 0.05, (H, W))).astype(np.float32)
        rgbs.append(x)
        rrefs.append(y)
        deps.append(d)
        drefs.append(dr)
    return rgbs, deps, rrefs, drefs


def _flat(lst):
    return torch.from_numpy(np.concatenate([a.reshape(-1) for a in lst])).cuda()


def _run(sizes, weights, seed=0, smooth=True, with_depth=True):
    rgbs, deps, rrefs, drefs = _views(sizes, seed, smooth)
    fn = gs.ImageLoss(sizes, weights)
    loss, d_rgb, d_depth = fn(_flat(rgbs), _flat(deps) if with_depth else None, _flat(rrefs),
                              _flat(drefs) if with_depth else None)
    torch.cuda.synchronize()
    ref = O.mapping_loss_views(rgbs, deps, rrefs, drefs, *weights)
    return loss.cpu().numpy().astype(np.float64), d_rgb.cpu().numpy(), d_depth.cpu().numpy(), ref, (rgbs, rrefs)


def _check_grad(got, ref_list, ssim_ref_list, rtol=1e-6):
    off = 0
    for g_ref, g_ssim in zip(ref_list, ssim_ref_list):
        n = g_ref.size
        g = got[off:off + n].reshape(g_ref.shape).astype(np.float64)
        tol = 1e-3 * np.abs(g_ssim).max() + rtol * np.abs(g_ref)
        err = np.abs(g - g_ref)
        assert (err <= tol).all(), "max err %g at tol %g" % (err.max(), tol[np.unravel_index(err.argmax(), err.shape)])
        off += n
    assert off == got.size


def _ssim_part(rgbs, rrefs, sizes, w_s):
    """The SSIM term's gradient alone (per view), from the oracle with the L1 weights at 0."""
    P = sum(W * H for W, H in sizes)
    out = []
    for x, y, (W, H) in zip(rgbs, rrefs, sizes):
        _, g, _ = O.mapping_loss(x, np.zeros((H, W)), y, np.zeros((H, W)), 0.0, 0.0, w_s)
        out.append(g * (W * H) / P)
    return out


@pytest.mark.parametrize("smooth", [True, False])
def test_eq3_loss_and_gradient_mixed_ragged_views(smooth):
    """Views of several sizes, none a multiple of the 32x16 tile; one smaller than the window."""
    sizes = [(64, 48), (37, 29), (100, 70), (5, 3)]
    loss, g_rgb, g_depth, ref, (rgbs, rrefs) = _run(sizes, gs.EQ3_WEIGHTS, seed=1, smooth=smooth)
    L, l1d, l1c, ss, gr, gd = ref
    np.testing.assert_allclose(loss, [L, l1d, l1c, ss], rtol=2e-5)
    _check_grad(g_rgb, gr, _ssim_part(rgbs, rrefs, sizes, 0.1))
    np.testing.assert_allclose(g_depth, np.concatenate([g.reshape(-1) for g in gd]), rtol=1e-6, atol=0)


def test_l1_only_weights_match_plain_means():
    """w = (0.1, 1/3, 0): mean L1 over RGB elements + 0.1 mean L1 depth; SSIM not computed (NaN)."""
    sizes = [(64, 48), (33, 17)]
    loss, g_rgb, g_depth, ref, _ = _run(sizes, gs.L1_WEIGHTS, seed=2)
    L, l1d, l1c, _, gr, gd = ref
    np.testing.assert_allclose(loss[:3], [L, l1d, l1c], rtol=2e-6)
    assert np.isnan(loss[3])
    np.testing.assert_allclose(g_rgb, np.concatenate([g.reshape(-1) for g in gr]), rtol=1e-6, atol=0)
    np.testing.assert_allclose(g_depth, np.concatenate([g.reshape(-1) for g in gd]), rtol=1e-6, atol=0)


def test_identical_images_give_zero_loss():
    sizes = [(48, 40)]
    rgbs, deps, _, _ = _views(sizes, 3)
    fn = gs.ImageLoss(sizes)
    x, d = _flat(rgbs), _flat(deps)
    loss, g_rgb, g_depth = fn(x, d, x.clone(), d.clone())
    torch.cuda.synchronize()
    assert abs(float(loss[0])) < 1e-6 and float(loss[3]) == pytest.approx(1.0, abs=1e-6)
    assert float(g_depth.abs().max()) == 0.0
    # SSIM is maximal there: its gradient vanishes up to rounding (scale w_s / (3 N_p) per unit dS)
    assert float(g_rgb.abs().max()) < 0.05 * 0.1 / (3 * 48 * 40)


def test_many_views_split_launches_and_no_depth():
    """70 views (more than one launch's 64) without depth (w_depth = 0); loss-only call agrees."""
    sizes = [(16, 12)] * 35 + [(9, 21)] * 35
    w = (0.0, 0.4, 0.1)
    loss, g_rgb, _, ref, (rgbs, rrefs) = _run(sizes, w, seed=4, with_depth=False)
    L, l1d, l1c, ss, gr, _ = ref
    np.testing.assert_allclose(loss[[0, 2, 3]], [L, l1c, ss], rtol=2e-5)
    assert loss[1] == 0.0
    _check_grad(g_rgb, gr, _ssim_part(rgbs, rrefs, sizes, 0.1))
    rgbs, deps, rrefs, drefs = _views(sizes, 4)
    fn = gs.ImageLoss(sizes, w)
    only, _, _ = fn(_flat(rgbs), None, _flat(rrefs), None, with_grad=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(only.cpu().numpy()[[0, 2, 3]], loss[[0, 2, 3]].astype(np.float32))


def test_deterministic():
    sizes = [(128, 96), (80, 60)]
    rgbs, deps, rrefs, drefs = _views(sizes, 5)
    fn = gs.ImageLoss(sizes)
    args = (_flat(rgbs), _flat(deps), _flat(rrefs), _flat(drefs))
    a = [t.clone() for t in fn(*args)]
    b = [t.clone() for t in fn(*args)]
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_full_size_640x480_view():
    """One 640x480 keyframe (the mapping workload's resolution), loss and a gradient sample."""
    sizes = [(640, 480)]
    loss, g_rgb, _, ref, (rgbs, rrefs) = _run(sizes, gs.EQ3_WEIGHTS, seed=6)
    L, l1d, l1c, ss, gr, _ = ref
    np.testing.assert_allclose(loss, [L, l1d, l1c, ss], rtol=2e-5)
    _check_grad(g_rgb, gr, _ssim_part(rgbs, rrefs, sizes, 0.1))


def test_autograd_function_backward():
    sizes = [(40, 30)]
    rgbs, deps, rrefs, drefs = _views(sizes, 7)
    fn = gs.ImageLoss(sizes)
    x = _flat(rgbs).requires_grad_(True)
    d = _flat(deps).requires_grad_(True)
    loss = gs.image_loss(x, d, _flat(rrefs), _flat(drefs), fn)
    (2.0 * loss).backward()
    L, _, _, _, gr, gd = O.mapping_loss_views(rgbs, deps, rrefs, drefs)
    assert float(loss.detach()) == pytest.approx(L, rel=2e-5)
    _check_grad(x.grad.cpu().numpy() / 2, gr, _ssim_part(rgbs, rrefs, sizes, 0.1))
    np.testing.assert_allclose(d.grad.cpu().numpy() / 2, gd[0].reshape(-1), rtol=1e-6)
