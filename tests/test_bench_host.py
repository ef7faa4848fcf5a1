"""Host-side arithmetic of bench.py (no GPU): tile specs, per-stage roofline fractions and the
per-view pixel mix, checked against hand-computed values."""
import importlib.util
import os
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_parse_tiles(bench):
    assert bench.parse_tiles("auto") is None
    assert bench.parse_tiles("80x60=8x8,320x240=32x16") == {(80, 60): (8, 8), (320, 240): (32, 16)}


def test_stage_roofline_fractions(bench):
    pipe = dict(pairs=1_000_000, records=10_000, contributing=2_000_000, pair_views=100_000)
    ms = {"gs_project": 1.0, "gs_bin_sort": 2.0, "gs_info_gain_composite": 4.0}
    out = bench.stage_roofline(pipe, ms, hbm_gbs=1000.0, issue_tps=10.0)
    # projection: (25 * 1e5 + 110 * 1e4) instr in 1 ms = 3.6e9 / s of 1e13
    assert out["gs_project"]["frac"] == pytest.approx(3.6e9 / 1e13)
    # binning: 44 B * 1e6 in 2 ms = 22 GB/s of 1000
    assert out["gs_bin_sort"]["achieved"] == pytest.approx(22.0) and out["gs_bin_sort"]["frac"] == pytest.approx(0.022)
    # compositing: 12 * 2e6 in 4 ms = 6e9 / s
    assert out["gs_info_gain_composite"]["frac"] == pytest.approx(6e9 / 1e13)
    assert bench.stage_roofline(pipe, {}, 1000.0, 10.0) == {}


def test_map_stage_roofline_fractions(bench):
    ws = dict(records=1000, pairs=50_000, evaluated=1_000_000, contributing=200_000, pixels=10_000)
    ms = {"gs_render_bwd": 1.0, "gs_image_loss": 0.5, "gs_adam_step": 0.25}
    out = bench.map_stage_roofline(ws, n=5_000, n_views=2, stage_ms=ms, hbm_gbs=1000.0, issue_tps=10.0)
    assert out["gs_render_bwd"]["frac"] == pytest.approx((10 * 1e6 + 38 * 2e5) / 1e-3 / 1e13)
    assert out["gs_image_loss"]["achieved"] == pytest.approx(12 * 4 * 1e4 / 0.5e-3 / 1e9)
    assert out["gs_adam_step"]["achieved"] == pytest.approx(28 * 16 * 5000 / 0.25e-3 / 1e9)
    assert "gs_project" not in out


def test_mix_pixels_per_view(bench):
    cams = [SimpleNamespace(width=80, height=60), SimpleNamespace(width=160, height=120),
            SimpleNamespace(width=320, height=240)]
    assert bench.mix_pixels_per_view(cams) == pytest.approx((4800 + 19200 + 76800) / 3)


def test_issue_peak_at_the_load_clock(bench):
    r = [{"bound": "alu", "achieved": 4.0}, {"bound": "hbm", "achieved": 1000.0}]
    bench.at_load_clock(r, 152, 2000.0)
    assert r[0]["peak_at_load_clock"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert r[0]["frac_at_load_clock"] == pytest.approx(4.0 / (152 * 128 * 2000e6 / 1e12))
    assert "peak_at_load_clock" not in r[1]
    assert bench.at_load_clock(r[1:], 152, None) == r[1:]


def test_headline_roofline_reproduces_from_its_fields(bench):
    """frac = 12 x contributing evaluations / launch time / (SMs x 128 x clock): the line's
    roofline can be recomputed from launch_ms, contributing_evals and the stated peak."""
    assert bench.IG_INSTR_PER_EVAL == 12.0
    contrib, launch_ms = 886_993_606, 3.106
    ach = bench.compositing_rate(contrib, launch_ms / 1e3)
    peak = 152 * 128 * 2070e6 / 1e12
    assert ach == pytest.approx(12 * contrib / (launch_ms / 1e3) / 1e12)
    assert ach / peak == pytest.approx(0.0851, abs=5e-4)
