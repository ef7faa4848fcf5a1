"""Writes oracle_tiny_scene.json: the FP64 oracle's results on a tiny seeded scene.

These are the oracle's own outputs, not the paper's: a regression fixture.  tests/test_golden.py
recomputes them with the oracle and compares, so that any change to the oracle's arithmetic
shows up as a fixture change that has to be regenerated on purpose (and justified by the
passage of the paper it follows).  Only the oracle and the seeded input generator are used.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O                       # noqa: E402
from paper_2409_18122_gb300 import scenes            # noqa: E402
from paper_2409_18122_gb300.scenes import Camera     # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny_scene.json")
SAMPLE_PIXELS = [(0, 0), (3, 5), (11, 16), (12, 31), (7, 7), (23, 0), (15, 15), (20, 9)]
SAMPLE_GAUSSIANS = [0, 3, 17, 42, 99, 150, 199]


def scene():
    """200 Gaussians uniform in [-2, 2]^2 x [1, 5] (seed 77); a 32x24 view with the default
    16x16 tiles and a 16x16 view with 8x8 tiles, both at the origin looking down +z."""
    g = scenes.random_scene(77, 200, [])
    cams = [Camera(40, 40, 16, 12, 32, 24), Camera(30, 30, 8, 8, 16, 16).with_tile(8, 8)]
    return g, cams


def compute():
    g, cams = scene()
    pr = O.project(g, cams)
    rec = O.records_from_projection(pr)
    b = O.bin_sort(rec, cams)
    ig, _ = O.info_gain(g, cams)
    imgs = O.render_images(g, cams)
    views = []
    for cam, im in zip(cams, imgs):
        H, W = cam.height, cam.width
        views.append({
            "sums": {"rgb": im["rgb"].sum(axis=(0, 1)).tolist(), "depth": float(im["depth"].sum()),
                     "unc": float(im["unc"].sum()), "T": float(im["T"].sum())},
            "last_id": im["last_id"].astype(np.int64).ravel().tolist(),
            "pixels": [{"yx": [y % H, x % W], "rgb": im["rgb"][y % H, x % W].tolist(),
                        "depth": float(im["depth"][y % H, x % W]), "unc": float(im["unc"][y % H, x % W]),
                        "T": float(im["T"][y % H, x % W])} for y, x in SAMPLE_PIXELS],
        })
    # gradient of the mean of all RGB values plus 0.1 x the mean depth
    dimg = []
    P = sum(c.width * c.height for c in cams)
    for cam in cams:
        d = np.zeros((cam.height, cam.width, 4))
        d[..., :3] = 1.0 / (3 * P)
        d[..., 3] = 0.1 / P
        dimg.append(d)
    gr = O.grad(g, cams, dimg)
    grads = {k: {"sum": np.asarray(v, np.float64).sum(axis=0).tolist(),
                 "rows": {str(i): np.asarray(v, np.float64)[i].tolist() for i in SAMPLE_GAUSSIANS}}
             for k, v in gr.items() if k in ("dmo", "dsu", "dq", "drgb")}
    return {
        "n_records": int(len(rec["gid"])),
        "n_pairs": int(b["n_pairs"]),
        "keys": [int(k) for k in b["keys"]],
        "vals": [int(v) for v in b["vals"]],
        "ranges": b["ranges"].astype(np.int64).tolist(),
        "info_gain": [float(x) for x in ig],
        "views": views,
        "grads": grads,
    }


def main():
    data = {"written_by": "tests/golden/make_golden.py (the FP64 oracle on a seeded scene)"}
    data.update(compute())
    with open(OUT, "w") as f:
        json.dump(data, f, separators=(",", ":"))
        f.write("\n")
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
