"""Writes tests/golden/oracle_regression_small.json by calling only the oracle.

The paper prints no worked numeric example, image or gradient, so this fixture is an
oracle regression record, not a paper value: a 12-Gaussian scene (inputs stored in the
file, so no random generator is re-run) rendered as K=2 subsets at 24x20 with the
local render (Eq. 3-4), the composition (Eq. 5) and the backward (Eq. 6-7).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402
from paper_2606_18588_gb300 import inputs as I  # noqa: E402


def case():
    rng = np.random.default_rng(1234)
    n = 12
    sc = I.Scene(rng.uniform(-0.4, 0.4, (n, 3)).astype(np.float32),
                 rng.normal(-2.7, 0.3, (n, 3)).astype(np.float32),
                 rng.standard_normal((n, 4)).astype(np.float32),
                 rng.normal(0.5, 1.0, n).astype(np.float32),
                 rng.normal(0.0, 0.5, (n, 4, 3)).astype(np.float32), 1)
    cam = I.pinhole(24, 20, 60.0, (0.2, -0.1, -2.0), (0.0, 0.0, 0.0), 0.01)
    return sc, np.array([0, 6, 12]), cam


def main():
    sc, off, cam = case()
    o = O.opts(tile=8)
    view = O.render_view(sc, off, cam, o)
    dLdC = np.ones((3, cam.height, cam.width))
    g = O.backward_view(sc, off, cam, dLdC, None, o)
    out = {
        "source": "oracle regression (make_golden.py); the paper prints no worked example",
        "inputs": {k: a.tolist() for k, a in zip(
            ["means", "log_scales", "quats", "opacity_logits", "sh"], sc.arrays())},
        "sh_degree": sc.sh_degree, "offsets": off.tolist(),
        "camera": {"R": cam.R.tolist(), "t": cam.t.tolist(), "fx": cam.fx, "fy": cam.fy,
                   "cx": cam.cx, "cy": cam.cy, "width": cam.width, "height": cam.height,
                   "near": cam.near},
        "image": view["image"].tolist(), "T": view["T"].tolist(),
        "grad_means": g[0].tolist(), "grad_opacity_logits": g[3].tolist(),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                           "oracle_regression_small.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
