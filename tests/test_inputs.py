"""The seeded synthetic inputs against the recipe they are documented with: sizes, camera
rigs, resolution mixes and the distributions of the Gaussian attributes.  The generators
hold none of the method's arithmetic; these checks keep the benchmark and the parity tests
on the workloads they claim."""
import numpy as np
import pytest

from paper_2409_18122_gb300 import scenes


def _level_rig(c):
    """Camera-to-world R of a level camera: down = -z_world, forward horizontal, right = down x forward."""
    R = np.asarray(c.R, np.float64)
    np.testing.assert_allclose(R[:, 1], [0, 0, -1], atol=1e-7)
    assert abs(R[2, 2]) < 1e-7
    np.testing.assert_allclose(R[:, 0], np.cross(R[:, 1], R[:, 2]), atol=1e-6)
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-6)


def _check_attributes(g, tol):
    ls, logit, rgb, u = g.su[:, :3], g.mo[:, 3], g.rgb[:, :3], g.su[:, 3]
    assert abs(ls.mean() + 3.0) < tol and abs(ls.std() - 0.5) < tol          # log-scales N(-3, 0.5)
    assert abs(logit.mean()) < 2 * tol and abs(logit.std() - 1.0) < 2 * tol  # opacity logit N(0, 1)
    assert rgb.min() >= 0 and rgb.max() <= 1 and abs(rgb.mean() - 0.5) < tol  # RGB U[0, 1]
    assert u.min() >= 0 and u.max() <= 1 and abs(u.mean() - 0.5) < tol        # uncertainty U[0, 1]
    np.testing.assert_allclose(np.linalg.norm(g.q.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert (g.rgb[:, 3] == 0).all()


def test_config0_small_case():
    sc = scenes.config0()
    assert sc.seed == 1000 and sc.gmap.n == 2000
    mu = sc.gmap.mo[:, :3]
    assert (mu[:, :2] >= -2).all() and (mu[:, :2] <= 2).all() and (mu[:, 2] >= 1).all() and (mu[:, 2] <= 5).all()
    (c,) = sc.cams
    assert (c.width, c.height, c.fx, c.fy, c.cx, c.cy) == (128, 96, 100.0, 100.0, 64.0, 48.0)
    np.testing.assert_array_equal(c.R, np.eye(3))
    np.testing.assert_array_equal(c.T, np.zeros(3))
    _check_attributes(sc.gmap, 0.05)
    again = scenes.config0()
    for a, b in zip(sc.gmap.arrays(), again.gmap.arrays()):
        np.testing.assert_array_equal(a, b)     # seeded: the same arrays every time


def test_room_patches_are_planar_squares():
    """Gaussians split evenly over 50 patches, each a square of side 0.5-2 m with N(0, 0.02 m)
    scatter along its normal: per patch, the smallest principal spread is the scatter and the
    in-plane extent at most half the largest side."""
    n, P = 20_000, 50
    mu = scenes.room_means(np.random.default_rng(7), n)
    per = n // P
    spreads, extents = [], []
    for k in range(P):
        x = mu[k * per:(k + 1) * per]
        x = x - x.mean(axis=0)
        _, s, vt = np.linalg.svd(x, full_matrices=False)
        spreads.append(s[-1] / np.sqrt(per))
        extents.append(np.abs(x @ vt[:2].T).max())
    assert 0.017 < np.median(spreads) < 0.023
    assert max(extents) < 1.0 * np.sqrt(2) + 0.1                 # half-diagonal of a 2 m square
    assert (mu > -1.5).all() and (mu[:, :2] < 11.5).all() and (mu[:, 2] < 4.5).all()


def test_keyframes_look_into_the_room():
    """cfg1 / cfg2 keyframes: 640x480, f = 525, centred principal point, positioned 0.5 m from
    the walls at 1-2 m height, heading within 45 degrees of the room centre."""
    for sc, n, V in ((scenes.config1(), 200_000, 1), (scenes.config2(), 500_000, 4)):
        assert sc.gmap.n == n and len(sc.cams) == V
        for c in sc.cams:
            assert (c.width, c.height, c.fx, c.fy, c.cx, c.cy) == (640, 480, 525.0, 525.0, 320.0, 240.0)
            _level_rig(c)
            x, y, z = c.T
            assert 0.5 <= x <= 9.5 and 0.5 <= y <= 9.5 and 1.0 <= z <= 2.0
            fwd = np.asarray(c.R, np.float64)[:2, 2]
            to_centre = np.array([5.0 - x, 5.0 - y])
            cosang = fwd @ to_centre / np.linalg.norm(fwd) / np.linalg.norm(to_centre)
            assert cosang >= np.cos(np.pi / 4) - 1e-6
    assert scenes.config1().seed == 1001 and scenes.config2().seed == 1002


def test_config3_candidate_lattice():
    """256 candidates on a 16 x 16 lattice (0.5 .. 9.5 m) at 1.5 m, resolutions by index mod 3
    (86 / 85 / 85), f = 0.8203 W, centred principal point, level cameras; 1M Gaussians."""
    sc = scenes.config3()
    assert sc.seed == 1003 and sc.gmap.n == 1_000_000 and len(sc.cams) == 256
    xs = np.linspace(0.5, 9.5, 16)
    res = [(80, 60), (160, 120), (320, 240)]
    for i, c in enumerate(sc.cams):
        np.testing.assert_allclose(c.T, [xs[i % 16], xs[i // 16], 1.5], atol=1e-6)
        assert (c.width, c.height) == res[i % 3]
        assert c.fx == pytest.approx(0.8203 * c.width, rel=1e-7) and c.fy == c.fx
        assert (c.cx, c.cy) == (c.width / 2, c.height / 2)
        _level_rig(c)
    counts = [sum((c.width, c.height) == r for c in sc.cams) for r in res]
    assert counts == [86, 85, 85]
    _check_attributes(sc.gmap, 0.005)


def test_config4_large_map():
    """3M Gaussians in a 40 x 40 x 3 m map, 8 keyframes 1280x720 (f = 1050), 1,024 candidates
    on a 32 x 32 lattice alternating 160x120 and 320x240."""
    sc, cands = scenes.config4()
    assert sc.seed == 1004 and sc.gmap.n == 3_000_000
    assert len(sc.cams) == 8 and all((c.width, c.height, c.fx) == (1280, 720, 1050.0) for c in sc.cams)
    assert len(cands) == 1024
    assert [(c.width, c.height) for c in cands[:4]] == [(160, 120), (320, 240)] * 2
    assert sum(c.width == 160 for c in cands) == 512
    xs = np.linspace(0.5, 39.5, 32)
    np.testing.assert_allclose(cands[33].T, [xs[1], xs[1], 1.5], atol=1e-5)
    mu = sc.gmap.mo[:, :3]
    assert mu[:, 0].max() > 35 and mu[:, 1].max() > 35      # spread over the whole 40 m map


def test_mapping_targets_are_perturbed_copies():
    sc = scenes.config0()
    t = scenes.perturbed(sc.gmap, seed=2002)
    d_mu = (t.mo[:, :3] - sc.gmap.mo[:, :3]).astype(np.float64)
    d_c = (t.rgb[:, :3] - sc.gmap.rgb[:, :3]).astype(np.float64)
    assert abs(d_mu.std() - 0.01) < 0.001 and abs(d_c.std() - 0.05) < 0.005
    np.testing.assert_array_equal(t.su, sc.gmap.su)
    np.testing.assert_array_equal(t.q, sc.gmap.q)
    np.testing.assert_array_equal(t.mo[:, 3], sc.gmap.mo[:, 3])
