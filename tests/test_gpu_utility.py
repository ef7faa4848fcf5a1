"""Render-free view utility (Sec. IV-A/B, Eq. view_util) through the C ABI vs the oracle.

Counts of visible high / low uncertainty Gaussians are integers decided in FP32 on both
sides (same operation sequence) and must match exactly; thresholds are FP64 (agree to
rounding); sums and region means are compared within FP32 tolerance."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2409_18122_gb300 import gs, scenes

pytestmark = pytest.mark.gpu


def _scene(n=20_000, n_side=4, seed=9):
    sc = scenes.config3(n=n, n_side=2)
    rng = np.random.default_rng(seed)
    cams = scenes.candidate_lattice(rng, n_side, 10.0, scenes.IG_RESOLUTIONS)
    return sc.gmap, cams


def _thr_gpu(gm, vu):
    st = vu.thresholds(gm).cpu().numpy()
    torch.cuda.synchronize()
    return st


def test_uncertainty_update_vs_oracle():
    rng = np.random.default_rng(1)
    n = 50_000
    prev = np.zeros((n, 4), np.float32)
    prev[:, :3] = rng.uniform(-5, 5, (n, 3))
    cur = prev.copy()
    moved = rng.uniform(size=n) < 0.7
    cur[moved, :3] += rng.normal(0, 0.05, (moved.sum(), 3)).astype(np.float32)
    su = np.zeros((n, 4), np.float32)
    su[:, 3] = rng.uniform(0, 1, n)
    for squared in (False, True):
        d_prev, d_cur = torch.from_numpy(prev).cuda(), torch.from_numpy(cur).cuda()
        d_su = torch.from_numpy(su).cuda()
        gs.uncertainty_update(d_prev, d_cur, d_su, squared=squared)
        got = d_su.cpu().numpy()
        ref = O.uncertainty_update(prev, cur, su[:, 3].astype(np.float64), squared=squared)
        np.testing.assert_array_equal(got[~moved, 3], su[~moved, 3])        # bookkeeping: kept bit for bit
        np.testing.assert_allclose(got[moved, 3], ref[moved], rtol=4e-7, atol=0)
        np.testing.assert_array_equal(got[:, :3], su[:, :3])


@pytest.mark.parametrize("ground_z", [float("-inf"), 0.3])
def test_thresholds_vs_oracle(ground_z):
    gmap, cams = _scene()
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    vu = gs.ViewUtility(cams, ground_z=ground_z)
    st = _thr_gpu(gm, vu)
    ref = O.uncertainty_thresholds(gmap.mo, gmap.su[:, 3], ground_z)
    assert st[4] == ref[4] and ref[4] > 0
    np.testing.assert_allclose(st[:4], ref[:4], rtol=1e-13, atol=0)


def _check_counts(gmap, cams, ground_z=float("-inf"), lam=1.0, range_m=5.0):
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    vu = gs.ViewUtility(cams, lam=lam, range_m=range_m, ground_z=ground_z)
    st = _thr_gpu(gm, vu)
    xi = vu(gm, gs.L.GS_XI).cpu().numpy()
    cnt = vu.counts.cpu().numpy().astype(np.int64)
    ref_xi, ref_cnt = O.view_utility(gmap.mo, gmap.su[:, 3], cams, range_m=range_m, lam=lam, ground_z=ground_z,
                                     thresholds=tuple(float(x) for x in st))
    # every Gaussian is far from both thresholds, so the FP64 classes are unambiguous
    u = gmap.su[:, 3].astype(np.float64)
    assert (np.abs(u - st[2]) > 1e-12 * abs(st[2])).all() and (np.abs(u - st[3]) > 1e-12 * abs(st[3])).all()
    np.testing.assert_array_equal(cnt, ref_cnt)
    np.testing.assert_array_equal(xi, ref_xi.astype(np.float32))
    return cnt


def test_view_utility_counts_bit_exact():
    gmap, cams = _scene()
    cnt = _check_counts(gmap, cams)
    assert cnt.sum() > 1000


def test_view_utility_lambda_range_ground():
    gmap, cams = _scene(n=30_000, seed=4)
    _check_counts(gmap, cams, ground_z=0.4, lam=0.5, range_m=3.0)


def test_view_utility_sum_mode():
    gmap, cams = _scene(seed=5)
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    vu = gs.ViewUtility(cams)
    xs = vu(gm, gs.L.GS_XI_SUM).cpu().numpy().astype(np.float64)
    ref, _ = O.view_utility(gmap.mo, gmap.su[:, 3], cams, mode="sum")
    np.testing.assert_allclose(xs, ref, rtol=2e-5, atol=1e-6)


def test_view_utility_deterministic_and_single_view_equal():
    gmap, cams = _scene(seed=6)
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    vu = gs.ViewUtility(cams)
    vu.thresholds(gm)
    a = vu(gm, gs.L.GS_XI_SUM).clone()
    b = vu(gm, gs.L.GS_XI_SUM).clone()
    assert torch.equal(a, b)
    one = gs.ViewUtility([cams[2]])
    assert float(one(gm, gs.L.GS_XI_SUM)[0]) == pytest.approx(float(a[2]), rel=1e-5)


def test_view_utility_full_size_config3():
    """1M room Gaussians, all 256 candidates in one call; 32 of them checked against the oracle."""
    sc = scenes.config3()
    gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
    vu = gs.ViewUtility(sc.cams)
    st = _thr_gpu(gm, vu)
    vu(gm, gs.L.GS_XI)
    cnt = vu.counts.cpu().numpy().astype(np.int64)
    pick = list(range(0, 256, 8))
    _, ref_cnt = O.view_utility(sc.gmap.mo, sc.gmap.su[:, 3], [sc.cams[v] for v in pick],
                                thresholds=tuple(float(x) for x in st))
    np.testing.assert_array_equal(cnt[pick], ref_cnt)


def test_region_uncertainty_vs_oracle():
    gmap, _ = _scene(n=40_000, seed=7)
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    omega, count = gs.region_uncertainty(gm, (0.0, 0.0, 0.0), gs.REGION_SIZE_M, (4, 4, 2))
    ref, ref_cnt = O.region_uncertainty(gmap.mo, gmap.su[:, 3], (0.0, 0.0, 0.0), 2.5, (4, 4, 2))
    np.testing.assert_array_equal(count.cpu().numpy(), ref_cnt)
    np.testing.assert_allclose(omega.cpu().numpy(), ref, rtol=1e-6, atol=0)


def test_trajectory_utility_vs_oracle():
    gmap, _ = _scene(n=30_000, seed=12)
    rng = np.random.default_rng(12)
    n_traj, n_states = 6, 4
    cams = []
    for t in range(n_traj):
        x, y = rng.uniform(2, 8, 2)
        yaw = rng.uniform(0, 2 * np.pi)
        for l in range(n_states):   # a short straight path with a slight turn
            cams.append(scenes.yaw_camera(x + 0.3 * l * np.cos(yaw), y + 0.3 * l * np.sin(yaw), 1.5,
                                          yaw + 0.1 * l, 160, 120, 131.25))
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    vu = gs.ViewUtility(cams)
    st = _thr_gpu(gm, vu)
    s, best = gs.trajectory_utility(vu, gm, n_traj, n_states)
    ref, ref_best = O.trajectory_utility(gmap.mo, gmap.su[:, 3], cams, n_traj, n_states,
                                         thresholds=tuple(float(x) for x in st))
    np.testing.assert_array_equal(s.cpu().numpy(), ref.astype(np.float32))
    assert int(best.item()) == ref_best


def test_collision_check_vs_oracle():
    gmap, _ = _scene(n=50_000, seed=13)
    rng = np.random.default_rng(13)
    pts = np.zeros((129, 4), np.float32)
    pts[:, :3] = rng.uniform([0, 0, 0.2], [10, 10, 2.5], (129, 3))
    gm = gs.GaussianMapTensors.from_numpy(gmap)
    for r_robot, lam, gz in ((0.25, 3.0, float("-inf")), (0.05, 1.0, 0.3)):
        margin, hit = gs.collision_check(gm, torch.from_numpy(pts).cuda(), r_robot, lam, gz)
        ref_m, ref_h = O.collision_check(gmap.mo, gmap.su, pts, r_robot, lam, gz)
        np.testing.assert_array_equal(hit.cpu().numpy().astype(bool), ref_h)
        np.testing.assert_allclose(margin.cpu().numpy(), ref_m, rtol=1e-5, atol=2e-6)
        assert 0 < ref_h.sum() < len(pts)
