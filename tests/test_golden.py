"""The parameters the paper prints (tests/golden/paper_parameters.txt, each line with its
citation) against the defaults of the library, the oracle and the benchmark workloads."""
import importlib.util
import inspect
import os

import numpy as np

from oracle import oracle as O
from paper_2409_18122_gb300 import gs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _paper_parameters():
    out = {}
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, cite = line.split(None, 2)
            assert cite.startswith(("Sec.", "Eq.", "Tab.", "Fig.")), "uncited value %s" % name
            out[name] = float(value)
    return out


PAPER = _paper_parameters()


def _default(fn, name):
    return inspect.signature(fn).parameters[name].default


def test_every_value_is_read():
    assert set(PAPER) == {"w_depth", "lambda_1", "lambda_2", "threshold_sigmas", "region_size_m",
                          "lambda_xi", "lambda_g", "collision_points"}


def test_eq3_weights():
    eq3 = (PAPER["w_depth"], PAPER["lambda_1"], PAPER["lambda_2"])
    assert gs.EQ3_WEIGHTS == eq3
    assert tuple(_default(O.mapping_loss, k) for k in ("w_d", "w_c", "w_s")) == eq3
    assert tuple(_default(O.mapping_loss_views, k) for k in ("w_d", "w_c", "w_s")) == eq3


def test_uncertainty_thresholds_half_a_sigma():
    """u = (1, 3): mean 2, population sigma 1, so the thresholds sit at 2 +- the printed factor."""
    mo = np.zeros((2, 4), np.float32)
    mean, sigma, t_hi, t_lo, m = O.uncertainty_thresholds(mo, np.array([1.0, 3.0], np.float32))
    assert (mean, sigma, m) == (2.0, 1.0, 2)
    assert t_hi == 2.0 + PAPER["threshold_sigmas"] and t_lo == 2.0 - PAPER["threshold_sigmas"]


def test_view_utility_and_collision_defaults():
    assert _default(gs.ViewUtility.__init__, "lam") == PAPER["lambda_xi"] == gs.LAMBDA_XI
    assert _default(O.view_utility, "lam") == PAPER["lambda_xi"]
    assert _default(gs.collision_check, "lambda_g") == PAPER["lambda_g"] == gs.LAMBDA_G
    assert _default(O.collision_check, "lambda_g") == PAPER["lambda_g"]


def test_region_size():
    assert gs.REGION_SIZE_M == PAPER["region_size_m"]


def test_collision_workload_point_count():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.COLLISION_POINTS == int(PAPER["collision_points"])



def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _compare(got, ref, path="fixture"):
    """Integers exactly; floats to 1e-12 relative (the oracle is FP64 with a fixed operation
    order; libm may differ in the last bit between machines)."""
    if isinstance(ref, dict):
        assert set(got) == set(ref), path
        for k in ref:
            _compare(got[k], ref[k], path + "." + k)
    elif isinstance(ref, list):
        assert len(got) == len(ref), path
        for i, (g, r) in enumerate(zip(got, ref)):
            _compare(g, r, "%s[%d]" % (path, i))
    elif isinstance(ref, int):
        assert got == ref, path
    else:
        assert abs(got - ref) <= 1e-12 * abs(ref) + 1e-15, (path, got, ref)


def test_oracle_reproduces_its_tiny_scene_fixture():
    """Regression fixture (written by tests/golden/make_golden.py from the oracle alone):
    pair keys, tile ranges and last contributors exactly, images, information gain and
    gradients to FP64 rounding.  A deliberate change to the oracle regenerates it."""
    import json
    ref = json.load(open(os.path.join(GOLDEN, "oracle_tiny_scene.json")))
    ref.pop("written_by")
    got = json.loads(json.dumps(_make_golden().compute()))
    _compare(got, ref)
    assert ref["n_pairs"] == len(ref["keys"]) > 100
